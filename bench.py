#!/usr/bin/env python
"""Benchmark of the loop-estimate path: deflated loop estimates per second at a 1e-10 true residual.

Headline workload (the largest single-GPU configuration of the method): 24^3 x 32 lattice
(5.3 M complex unknowns), seeded near-identity SU(3) links with the spread tuned to a mean
plaquette of 0.600 (eps = 0.4323, seed 7; recon-12 link storage in the inner operator),
kappa = 0.157, 100 Z(4) noises, Q = 200 deflation eigenvectors of M' = M gamma_5 from one
MINRES-DR(240,200) super-convergence solve (the Hermitian path: the same space accelerates every
noise solve, M' y = eta by GMRES-Proj, x = gamma_5 y), 7-term PS and degree-6 POLY, all six
subtraction modes x nine operators, HFES projections on the tcgen05 tensor cores (split-precision
FP64).  Noise solves: FP16 storage of the inner Krylov basis with FP32 arithmetic inside an FP64
defect-correction loop that stops on the FP64 true residual <= 1e-10 (BF16 and plain FP64 are
measured on the same setup beside it).

The setup of the configuration (MINRES-DR, Min-Res coefficients, hopping traces by probing, 1/xi',
add-backs, tensor-core slices of the 200 vectors) runs once before the timed region and is
reported separately (setup_s) and amortised over the 100 noises (amortised_estimates_per_s).  One
step = the noise phase of one block of 10 noises (solves, the six subtraction vectors, the nine
contractions per timeslice); value = noises of all ranks / device time of the timed steps.

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

# headline workload
DIMS = (24, 24, 24, 32)
KAPPA = 0.157
LINK_EPS, LINK_SEED, NOISE_SEED = 0.4323, 7, 1
NNOISE, BLOCK = 100, 10
M_DR, K_DR, M_INNER = 240, 200, 40
HEAD_M_INNER = 100        # GMRES-Proj cycle length of the headline's FP16 / BF16 noise solves
INNER_WINDOW = 2          # Lanczos window of their inner cycles (M' is Hermitian)
INNER_TOL = 0.1            # inner (FP16 / BF16) GMRES-Proj stopping point inside the FP64 defect correction
K_PS, NPOLY = 7, 6
TOL, TOL_SPECIAL = 1e-10, 1e-12
MAX_CYCLES = 400
PREC_DEGREE = 0            # polynomial preconditioning of the noise solves (Krylov on M' p(M'))
WORKLOAD = ("24^3x32 kappa 0.157 (plaquette 0.600), 100 Z4 noises in steps of 10, MINRES-DR(240,200) on M gamma_5, "
            "Q=200, GMRES-Proj(100) noise solves in FP16 storage / FP32 arithmetic (Lanczos window 2 on the Hermitian "
            "M', inner "
            "tol 0.1) inside FP64 defect correction to 1e-10, PS K=7, POLY n=6, HFES on tensor cores, 6 modes x 9 "
            "operators")
# secondary: the 8^3 x 16 plain-FP64 workload (full loop estimate per step)
DIMS2 = (8, 8, 8, 16)
KAPPA2, NNOISE2, M2, K2, PLAQ2, SEED2 = 0.157, 50, 60, 30, 0.6, 2024
FP64_PEAK_TFLOPS = 152 * 2 * 2 * 2.07e9 / 1e12   # 2 DFMA / clock / SM at the 2070 MHz maximum clock
WILSON_FLOPS = 1368        # per site per right-hand side (1320 for P, 48 for 1 - kappa P)
L2_FLUSH_BYTES = 512 << 20
# DRAM bytes (read + write) per algorithmic byte of a kernel class, from an ncu capture of the same
# kernels on the 16^3 x 32 noise block (bench.py --case noise-block-f16)
DRAM_PER_ALGORITHMIC = {"dot": (1.017, "ncu dram__bytes_read.sum + dram__bytes_write.sum over 224 launches of "
                                       "multidot_kernel<__half2> on 16^3x32 / their algorithmic bytes"),
                        "wilson": (0.952, "ncu dram__bytes_read.sum + dram__bytes_write.sum of one launch of "
                                          "wilson_pair_kernel on FP16 fields, 24^3x32, 8 right-hand sides, recon 12 "
                                          "(405.0 MB) / its algorithmic bytes (425 MB)")}
# per-noise matrix-vector products of the plain FP64 noise solves on the headline workload (GPU
# path; the oracle runs the same algorithm): used to extrapolate the oracle's bounded sample
MATVECS_PER_NOISE_FP64 = 650


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=6)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="gb300", choices=["gb300", "reference"])
    ap.add_argument("--e2e-steps", type=int, default=None)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-dslash", action="store_true")
    ap.add_argument("--no-defl", action="store_true")
    ap.add_argument("--no-cfg2", action="store_true")
    ap.add_argument("--no-cfg35", action="store_true", help="skip the 16^3x32 and 12^3x24 derivative lines")
    ap.add_argument("--batch", action="store_true", help="also measure the uneven multi-lattice batch")
    ap.add_argument("--prec-degree", type=int, default=PREC_DEGREE,
                    help="degree of the polynomial preconditioner of the noise solves (0 = none)")
    ap.add_argument("--case", default=None,
                    choices=["gmres-cycle", "gmres-cycle-f32", "dslash-packed", "dslash-half", "defl-tensor",
                             "noise-block-f16"],
                    help="run one small kernel case for profiling instead of the benchmark")
    return ap.parse_args()


def dist_env():
    return int(os.environ.get("RANK", 0)), int(os.environ.get("WORLD_SIZE", 1)), int(os.environ.get("LOCAL_RANK", 0))


def link_seed(rank):
    """Seed of the gauge configuration of a rank: every rank works on its own configuration."""
    return LINK_SEED + rank


def make_links(rank):
    from paper_1903_06986_gb300 import synth
    return synth.su3_links(DIMS, LINK_EPS, link_seed(rank))


def reduce_max_over_ranks(t, world, device):
    """The largest t over the ranks of the job (t itself on one rank): a timed region ends when its
    slowest rank ends.  device: where the collective's tensor lives ("cuda" for NCCL, "cpu" for gloo)."""
    if world <= 1:
        return t
    import torch
    import torch.distributed as dist
    v = torch.tensor([float(t)], dtype=torch.float64, device=device)
    dist.all_reduce(v, op=dist.ReduceOp.MAX)
    return float(v.item())


def job_rate(units_per_rank, world, t_max):
    """Whole-job throughput: the units all ranks processed over the slowest rank's time."""
    return units_per_rank * world / t_max


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
    """Time the oracle on a bounded sample of the headline workload and extrapolate to estimates/s.

    Sample on 24^3 x 32 (about 20 s on the host): one Wilson operator application, one classical
    Gram-Schmidt pass (inner products and update) of a field against 8 basis fields, and the nine
    contractions of one noise.  Model of the oracle's own algorithm (the same as the GPU path's):
    per noise MATVECS_PER_NOISE_FP64 operator applications, each with CGS2 against on average 20
    GMRES-Proj(40) basis fields plus the projection over the 201-vector space once per 40 steps,
    then 12 subtraction matvecs, the projection over 200 vectors twice and 6 x 9 contractions;
    setup = MINRES-DR(240,200) (about 600 matvecs with CGS2 against on average 220 fields, and one
    241 x 201 basis rotation per 40 matvecs) plus the hopping traces (12 x 512 probes x 6 hops)."""
    from oracle import lattice as L, operators as O, rng
    t_start = time.perf_counter()
    eta = rng.z4_noise(NOISE_SEED, 0, DIMS)
    t0 = time.perf_counter()
    w = L.wilson(U, KAPPA, eta)
    t_w = time.perf_counter() - t0
    nb = 8
    Vb = np.stack([L.flat(np.roll(w, i, axis=0)) for i in range(nb)], axis=1)
    Vb /= np.linalg.norm(Vb, axis=0, keepdims=True)
    f = L.flat(eta).astype(np.complex128)
    t0 = time.perf_counter()
    h = Vb.conj().T @ f
    f = f - Vb @ h
    t_orth_vec = (time.perf_counter() - t0) / nb           # per basis field, one pass
    t0 = time.perf_counter()
    O.per_t(O.densities(U, KAPPA, eta, w))
    t_con = time.perf_counter() - t0
    per_mv = t_w + 2 * t_orth_vec * (20 + 201.0 / 40)     # CGS2: two passes
    per_noise = MATVECS_PER_NOISE_FP64 * per_mv + 12 * t_w + 2 * 200 * t_orth_vec + 6 * t_con
    setup = 600 * (t_w + 2 * t_orth_vec * 220) + 15 * 241 * 201 * t_orth_vec / 2 + 12 * 512 * 6 * t_w
    rate = NNOISE / (setup + NNOISE * per_noise)
    sample = ("oracle on 24^3x32, bounded sample (%.1f s): one Wilson application %.2f s, one Gram-Schmidt pass "
              "%.3f s per basis field (8 fields), nine contractions %.2f s; extrapolated with the method's counts "
              "(%d matvecs per noise with CGS2 over ~25 fields each, 12 subtraction matvecs, 2 projections over 200 "
              "vectors, 6 x 9 contractions; setup MINRES-DR(240,200) ~600 matvecs, 15 basis rotations, 36864 "
              "probe hops): rate = 100 / (setup + 100 x per-noise)"
              % (time.perf_counter() - t_start, t_w, t_orth_vec, t_con, MATVECS_PER_NOISE_FP64))
    return rate, sample, time.perf_counter() - t_start


def oracle_sample_threads(threads, timeout=600):
    """The same bounded oracle sample in a child process whose BLAS / OpenMP pools are limited to
    `threads` (set before numpy loads): (rate, seconds), or None if the child failed."""
    code = ("import sys, json; sys.path.insert(0, %r); import bench; "
            "r, s, dt = bench.oracle_sample(bench.make_links(0)); print(json.dumps([r, dt]))" % ROOT)
    env = dict(os.environ)
    for var in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS", "BLIS_NUM_THREADS"):
        env[var] = str(threads)
    try:
        p = subprocess.run([sys.executable, "-c", code], env=env, capture_output=True, text=True, timeout=timeout)
        rate, dt = json.loads(p.stdout.strip().splitlines()[-1])
        return float(rate), float(dt)
    except Exception:
        return None


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
    U = make_links(0)
    times, rates = [], []
    sample = ""
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
            "config": {"workload": WORKLOAD, "lattice": "24x24x24x32", "noises": NNOISE},
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
    CUDA events on the library stream around each of 5 timed launches (after 2 warm-up ones), with
    L2 flushed before each (a 512 MB buffer written), so that links and fields come from DRAM as
    they do inside a solver, where the Gram-Schmidt streams evict them between applications."""
    from paper_1903_06986_gb300 import lqcd, synth
    ctx = lqcd.Context(DSLASH_DIMS, recon=12)
    V = int(np.prod(DSLASH_DIMS))
    U = torch.from_numpy(synth.su3_links(DSLASH_DIMS, 0.4323, 7)).cuda()
    packed_links = {12: ctx.pack_links_f32(U, 12), 18: ctx.pack_links_f32(U, 18)}
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.int32, device="cuda")
    out = {}
    cases = [("f64", 18, 1, 0), ("f64", 18, 8, 0), ("f32packed", 12, 1, 1), ("f32packed", 12, 8, 2),
             ("f32packed", 12, 16, 2), ("f32packed", 18, 8, 2), ("f16packed", 12, 1, 1), ("f16packed", 12, 8, 2),
             ("f16packed", 12, 16, 2), ("bf16packed", 12, 8, 2),
             ("f32packed", 12, 8, 3), ("f32packed", 12, 16, 3), ("f16packed", 12, 8, 3), ("f16packed", 12, 16, 3),
             ("bf16packed", 12, 8, 3), ("bf16packed", 12, 16, 3)]
    for prec, recon, nrhs, nr in cases:
        ctx.set_rhs_per_thread(nr)
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
            fn = lambda: ctx.wilson_apply_packed(Up, recon, 0.157, x, y, rhs_per_thread=nr)
            w, lreals = 4, recon
        for _ in range(2):
            fn()
        t = 0.0
        for _ in range(5):
            flush.fill_(1)
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            fn()
            e1.record()
            torch.cuda.synchronize()
            t += e0.elapsed_time(e1) / 1000.0
        t /= 5
        nbytes = nrhs * V * 48 * w + V * 4 * lreals * lw
        gbs = nbytes / t / 1e9
        tf = 1368.0 * V * nrhs / t / 1e12
        key = "%s_recon%d_rhs%d" % (prec, recon, nrhs) + ("_staged" if nr == 3 else "")
        out[key] = {
            "ms": round(t * 1e3, 4), "GB/s": round(gbs, 1), "TFLOP/s": round(tf, 4),
            "frac_hbm": round(gbs / HBM_PEAK_GBS, 4),
            "frac_fp64": round(tf / FP64_PEAK_TFLOPS, 4) if prec == "f64" else None}
        del x, y
    ctx.close()
    return {"lattice": "24x24x24x32", "bytes": "nrhs*V*24 reals read+written + links once",
            "l2": "flushed before every timed launch", "hbm_peak_gbs": HBM_PEAK_GBS, "results": out}


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
        eps = synth.eps_for_plaquette(dims, PLAQ2, SEED2 + 10 + i)
        U = torch.from_numpy(synth.su3_links(dims, eps, SEED2 + 10 + i)).cuda()
        probs.append(dict(ctx=lqcd.Context(dims, recon=12), links=U, kappa=BATCH_KAPPA, seed=NOISE_SEED,
                          nnoise=BATCH_NOISE, block=0, m=M2, k=K2, K=K_PS, npoly=NPOLY, tol=TOL,
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
    of the 8^3x16 workload (FP64, or the mixed solver's FP32 cycle), four applications of the
    packed FP32 or FP16 operator (recon 12, 8 right-hand sides) on the 24^3x32 lattice, the HFES
    projection on the tensor cores, or one FP16 noise block of the headline's method on 16^3x32."""
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
    if args.case == "noise-block-f16":
        # the headline's noise phase on a smaller lattice (16^3 x 32, kappa 0.157, Hermitian path with a
        # MINRES-DR(60,30) space, GMRES-Proj(100) with the Lanczos window): one block of 10 noises in FP16
        # storage; about 4 GB on the device
        dims = (16, 16, 16, 32)
        ctx = lqcd.Context(dims, recon=12)
        ctx.set_inner_window(INNER_WINDOW)
        U = torch.from_numpy(synth.su3_links(dims, LINK_EPS, LINK_SEED)).cuda()
        loop = ctx.loop_setup(U, KAPPA, NOISE_SEED, 10, 10, 60, 30, K_PS, NPOLY, TOL, TOL_SPECIAL, m_inner=HEAD_M_INNER,
                              max_cycles=MAX_CYCLES, prec=lqcd.PREC_F16, system=lqcd.SYS_MG5, inner_tol=INNER_TOL)
        torch.cuda.synchronize()
        setup_launches = ctx.launches
        per, ni = loop.noises(U, 0, 10)
        torch.cuda.synchronize()
        print(json.dumps({"case": args.case, "matvecs": ni["matvecs"], "setup_launches": setup_launches,
                          "launches": ctx.launches}))
        return
    dims2 = DIMS2
    U = torch.from_numpy(synth.su3_links(dims2, 0.4323, SEED2)).cuda()
    ctx = lqcd.Context(dims2)
    etas = ctx.noise_z4(NOISE_SEED, 0, NNOISE2)
    if args.case == "gmres-cycle":
        x, info, _ = ctx.gmresdr_solve(U, KAPPA2, etas, M2 - K2, 0, 1e-30, 1)
    else:
        _, _, defl = ctx.gmresdr_solve(U, KAPPA2, etas[:1].contiguous(), M2 - K2, 4, 1e-3, 5, want_defl=True)
        x, info = ctx.proj_solve(U, KAPPA2, defl, etas, M2 - K2, 1e-6, 1, prec=1)
    torch.cuda.synchronize()
    print(json.dumps({"case": args.case, "matvecs": info["matvecs"], "launches": ctx.launches}))


def cfg2_fp64(torch):
    """The plain-FP64 8^3 x 16 workload: one complete loop estimate per step at kappa = 0.157 (50
    noises, GMRES-DR(60,30) on M for GMRES-Proj and MINRES-DR(60,30) on M' for 30 HFES eigenpairs,
    PS K = 7, POLY n = 6, six modes); 1 warm-up and 2 timed steps, CUDA events on the library's
    stream; FP64 roofline of its dominant kernel class (FP64 pipe: 2 DFMA / clock / SM)."""
    from paper_1903_06986_gb300 import lqcd, synth
    eps = synth.eps_for_plaquette(DIMS2, PLAQ2, SEED2)
    U = torch.from_numpy(synth.su3_links(DIMS2, eps, SEED2)).cuda()
    ctx = lqcd.Context(DIMS2, recon=12)
    run = lambda: ctx.loop_estimate(U, KAPPA2, NOISE_SEED, NNOISE2, NNOISE2, M2, K2, K_PS, NPOLY, TOL, TOL_SPECIAL,
                                    max_cycles=1000)
    run()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    res = [run() for _ in range(2)]
    e1.record()
    torch.cuda.synchronize()
    t = e0.elapsed_time(e1) / 1000.0
    if not all(r["converged"] and r["max_true_resid"] <= TOL for r in res):
        raise RuntimeError("8^3x16 loop estimate did not reach the tolerance")
    ctx.timing(True)
    ctx.timing_reset()
    run()
    tm = ctx.timing_read()
    ctx.timing(False)
    flops_per_unit = {"wilson": WILSON_FLOPS, "dot": 8.0, "axpy": 8.0, "combine": 8.0, "norm": 4.0}
    dom = max(tm, key=lambda k: tm[k][0])
    ms, nl, units = tm[dom]
    fpu = flops_per_unit.get(dom)
    ach = units * fpu / (ms / 1000.0) / 1e12 if fpu and ms > 0 else None
    out = {"workload": "8^3x16 plain FP64, kappa 0.157, 50 Z4 noises, GMRES-DR(60,30)+MINRES-DR(60,30), Q=30, "
                       "PS K=7, POLY n=6, 6 modes x 9 operators; one complete loop estimate (setup included) per step",
           "value": 2 * NNOISE2 / t, "unit": "estimates/s", "ms_per_step": 1000.0 * t / 2,
           "setup_s": float(np.mean([r["seconds_setup"] for r in res])),
           "noise_phase_estimates_per_s": NNOISE2 * 2 / sum(r["seconds_noise"] for r in res),
           "roofline": {"kernel": dom, "bound": "alu", "achieved": ach, "peak": FP64_PEAK_TFLOPS, "unit": "TFLOP/s",
                        "frac": ach / FP64_PEAK_TFLOPS if ach else None,
                        "peak_source": "FP64 pipe: 152 SMs x 2 DFMA/clk x 2 flop x 2.07 GHz (derived)"},
           "breakdown_ms": {k: round(v[0], 1) for k, v in tm.items() if v[0] > 0}}
    ctx.close()
    return out


CFG3_DIMS = (16, 16, 16, 32)
CFG3_M, CFG3_K = 200, 160
CFG3_NOISE, CFG3_TIMED = 200, 64


def cfg3_batching(torch):
    """The 16^3 x 32 multi-right-hand-side workload in plain FP64: kappa 0.157, links of the main
    generator at plaquette 0.6, 160 eigenvectors from one MINRES-DR(200,160) run on M' = M gamma_5
    (GMRES-DR on M stagnates beyond this field's critical kappa), the 200 noises' block width picked
    by the autotuner among 8, 16, 32 and 64.  Timed: the first 64 noises (whole blocks of the chosen
    width), CUDA events on the library's stream; the rate of the other 136 is the same per noise."""
    from paper_1903_06986_gb300 import lqcd, synth
    U = torch.from_numpy(synth.su3_links(CFG3_DIMS, LINK_EPS, LINK_SEED + 1)).cuda()
    ctx = lqcd.Context(CFG3_DIMS, recon=12)
    ctx.set_defl_engine(lqcd.DEFL_TENSOR)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    loop = ctx.loop_setup(U, KAPPA, NOISE_SEED, CFG3_NOISE, 0, CFG3_M, CFG3_K, K_PS, NPOLY, TOL, TOL_SPECIAL,
                          m_inner=M_INNER, max_cycles=MAX_CYCLES, prec=lqcd.PREC_F64, system=lqcd.SYS_MG5)
    torch.cuda.synchronize()
    setup_s = time.perf_counter() - t0
    info = loop.info()
    bw = info["block"]
    loop.noises(U, 0, bw)  # warm-up: workspace and graphs at the chosen width
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    ntimed = max(bw, CFG3_TIMED // bw * bw)
    e0.record()
    stats = [loop.noises(U, first, bw)[1] for first in range(0, ntimed, bw)]
    e1.record()
    torch.cuda.synchronize()
    t = e0.elapsed_time(e1) / 1000.0
    if not all(s["converged"] and s["max_true_resid"] <= TOL for s in stats):
        raise RuntimeError("16^3x32 noise solves did not reach the tolerance")
    out = {"workload": "16^3x32 plain FP64, kappa 0.157 (plaquette 0.600), 200 Z4 noises in autotuned blocks, "
                       "MINRES-DR(200,160) on M gamma_5, Q=160, GMRES-Proj(40) to 1e-10, PS K=7, POLY n=6, 6 modes",
           "value": ntimed / t, "unit": "estimates/s", "noises_timed": ntimed,
           "autotuned_block": bw, "block_candidates": [8, 16, 32, 64], "Q": info["Q"],
           "setup_s": setup_s, "setup_matvecs": info["matvecs_setup"], "eig_resid_max": info["eig_resid_max"],
           "amortised_estimates_per_s": CFG3_NOISE / (setup_s + CFG3_NOISE * t / ntimed),
           "matvecs_per_noise": sum(s["matvecs"] for s in stats) / ntimed,
           "max_true_resid": max(s["max_true_resid"] for s in stats)}
    loop.close()
    ctx.close()
    return out


CFG5_DIMS = (12, 12, 12, 24)
CFG5_KAPPA, CFG5_NOISE, CFG5_BLOCK = 0.155, 64, 16
CFG5_M, CFG5_K = 80, 40
CFG5_H = 1e-5


def cfg5_derivs(torch):
    """The 12^3 x 24 differentiation workload: d Tr(Theta M^{-1}) / dkappa of the nine operators (NS
    and PS) and the link gradient of the NS scalar estimate, 64 noises, kappa 0.155, a MINRES-DR(80,40)
    space of M' (40 vectors) for the GMRES-Proj solves, in plain FP64 and in FP16 / FP32 mixed
    precision (3 solves per noise, 1e-10).  Check: a central difference (h = 1e-5) of the NS and PS
    loop estimates over the same noises against the FP64 d/dkappa."""
    from paper_1903_06986_gb300 import lqcd, synth
    U = torch.from_numpy(synth.su3_links(CFG5_DIMS, LINK_EPS, LINK_SEED + 2)).cuda()
    ctx = lqcd.Context(CFG5_DIMS, recon=12)
    args = (NOISE_SEED, CFG5_NOISE, CFG5_BLOCK, CFG5_M, CFG5_K, K_PS, TOL, TOL_SPECIAL)
    run = lambda prec: lqcd.loop_derivs(ctx, U, CFG5_KAPPA, *args, m_inner=M_INNER, max_cycles=MAX_CYCLES,
                                        prec=prec, system=lqcd.SYS_MG5)
    out = {"workload": "12^3x24 kappa 0.155, 64 Z4 noises in blocks of 16, MINRES-DR(80,40) on M gamma_5, "
                       "GMRES-Proj(40) x 3 solves per noise to 1e-10; d/dkappa of 9 operators (NS, PS K=7) and "
                       "the link gradient of the NS scalar estimate (setup included)"}
    res = {}
    for name, prec in (("fp16", lqcd.PREC_F16), ("fp64", lqcd.PREC_F64)):
        if prec != lqcd.PREC_F64:
            run(prec)  # warm-up (the FP64 run, after it, finds the context's workspace made)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        r = run(prec)
        torch.cuda.synchronize()
        t = time.perf_counter() - t0
        if not r["converged"] or r["max_true_resid"] > TOL:
            raise RuntimeError("derivative solves did not reach the tolerance")
        res[name] = r
        out[name] = {"value": CFG5_NOISE / t, "unit": "noise derivatives/s", "s": t, "matvecs": r["matvecs"]}
    d64, d16 = res["fp64"], res["fp16"]
    g64, g16 = d64["link_grad"].cpu().numpy(), d16["link_grad"].cpu().numpy()
    out["fp16_vs_fp64"] = {
        "dkappa_max_rel_diff": float((np.abs(d16["dkappa"] - d64["dkappa"]) /
                                      np.maximum(np.abs(d64["dkappa"]), 1e-300)).max()),
        "link_grad_rel_diff": float(np.linalg.norm(g16 - g64) / np.linalg.norm(g64))}
    # central difference of the estimates themselves (same noises, solves to 1e-12)
    kw = dict(m=CFG5_M, k=CFG5_K, K=K_PS, npoly=NPOLY, tol=1e-12, tol_special=1e-12, m_inner=M_INNER,
              max_cycles=MAX_CYCLES, system=lqcd.SYS_MG5, modes=lqcd.SUB_NONE | lqcd.SUB_PERT)
    f = {sg: ctx.loop_estimate(U, CFG5_KAPPA + sg * CFG5_H, NOISE_SEED, CFG5_NOISE, CFG5_BLOCK, **kw)["mean"]
         for sg in (-1, 1)}
    fd = (f[1] - f[-1]) / (2 * CFG5_H)
    rel = [float(np.max(np.abs(d64["dkappa"][m] - fd[m]) / np.maximum(np.abs(fd[m]), 1e-300))) for m in range(2)]
    out["dkappa_vs_central_difference"] = {"h": CFG5_H, "max_rel_diff_ns": rel[0], "max_rel_diff_ps": rel[1]}
    ctx.close()
    return out


def _block_first(i):
    """First noise of step i: the steps run through the 100 noises in blocks of BLOCK, cyclically."""
    return (BLOCK * i) % NNOISE


def _estimates(per, info_add):
    """Per-noise estimates [6][n][9] from noise terms [6][n][9][Lt] and add-backs [6][9][Lt]."""
    return per.sum(axis=-1) + info_add.sum(axis=-1)[:, None, :]


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

    def barrier():
        if world > 1:
            torch.distributed.barrier()
        torch.cuda.synchronize()

    def max_over_ranks(t):
        return reduce_max_over_ranks(t, world, "cuda")

    U = make_links(rank)
    ctx = lqcd.Context(DIMS, recon=12)        # the synthetic links are SU(3)
    Ud = torch.from_numpy(U).cuda()
    ctx.set_defl_engine(lqcd.DEFL_TENSOR)
    ctx.set_inner_window(INNER_WINDOW)

    # ---- setup of the configuration, once (reported separately, amortised below)
    barrier()
    t0 = time.perf_counter()
    loop = ctx.loop_setup(Ud, KAPPA, NOISE_SEED, NNOISE, BLOCK, M_DR, K_DR, K_PS, NPOLY, TOL, TOL_SPECIAL,
                          m_inner=HEAD_M_INNER, max_cycles=MAX_CYCLES, prec=lqcd.PREC_F16, system=lqcd.SYS_MG5,
                          inner_tol=INNER_TOL,
                          prec_degree=args.prec_degree)
    barrier()
    setup_s = time.perf_counter() - t0
    info = loop.info()
    add = info["addback"]
    outputs = {}

    def step(i, prec_name, host_links=None):
        first = _block_first(i)
        if host_links is None:
            per, ni = loop.noises(Ud, first, BLOCK)
        else:
            per, ni = loop.noises_host(host_links, first, BLOCK)
        if not ni["converged"] or ni["max_true_resid"] > TOL:
            raise RuntimeError("noise solves did not reach the tolerance: %g" % ni["max_true_resid"])
        outputs[(prec_name, first)] = per
        return ni

    # ---- headline: FP16 noise phase, device-resident inputs
    for i in range(args.warmup):
        step(i, "fp16")
    clocks = Clocks(local)
    barrier()
    clocks.start()
    launches0 = ctx.launches
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    stats = []
    ev0.record()
    for i in range(args.steps):
        stats.append(step(args.warmup + i, "fp16"))
    ev1.record()
    barrier()
    t_dev = ev0.elapsed_time(ev1) / 1000.0
    clk = clocks.stop()
    launches = ctx.launches - launches0
    t_max = max_over_ranks(t_dev)
    value = job_rate(BLOCK * args.steps, world, t_max)
    per_noise_s = t_max / (BLOCK * args.steps)

    # ---- kernel-class breakdown of one more step (per-launch events on; not part of the value)
    ctx.timing(True)
    ctx.timing_reset()
    step(args.warmup + args.steps, "fp16")
    tm = ctx.timing_read()
    tbytes = ctx.timing_bytes()
    ctx.timing(False)

    # ---- BF16 and plain FP64 noise phases on the same setup, and the per-estimate differences
    loop.set_noise_opts(lqcd.PREC_BF16, INNER_TOL)
    step(0, "bf16")
    nb16 = 3
    barrier()
    b0 = time.perf_counter()
    for i in range(nb16):
        step(1 + i, "bf16")
    barrier()
    t_bf16 = max_over_ranks(time.perf_counter() - b0)
    # plain FP64 at its own measured cycle length (GMRES-Proj(40), two Gram-Schmidt passes)
    loop.set_noise_opts(lqcd.PREC_F64)
    loop.set_inner_restart(M_INNER)
    barrier()
    f0 = time.perf_counter()
    step(0, "fp64")
    barrier()
    t_fp64 = max_over_ranks(time.perf_counter() - f0)
    loop.set_inner_restart(HEAD_M_INNER)
    loop.set_noise_opts(lqcd.PREC_F16, INNER_TOL)
    est64 = _estimates(outputs[("fp64", 0)], add)
    lam_min = float(np.abs(info["lam"]).min())
    nrm_eta2 = 12.0 * np.prod(DIMS)
    # two solutions with relative residuals <= tol differ by at most 2 tol ||eta|| / sigma_min(M), and
    # |Theta| <= 2 for these operators: |Delta estimate| <= 4 tol ||eta||^2 / sigma_min, sigma_min(M) =
    # smallest |lambda'| of the Hermitian M' = M gamma_5 (its smallest singular value)
    bound = 4.0 * TOL * nrm_eta2 / lam_min
    errors = {}
    for name in ("fp16", "bf16"):
        if (name, 0) in outputs:
            d = np.abs(_estimates(outputs[(name, 0)], add) - est64)
            errors[name] = {"max_abs_diff": float(d.max()),
                            "max_rel_diff": float((d / np.maximum(np.abs(est64), 1e-300)).max()),
                            "stated_bound_abs": bound}

    # ---- end to end through the public API: the C-ABI call takes the links in pinned host memory and
    # copies them to the device every step; the per-noise results return to host memory in the call
    e2e_steps = args.e2e_steps if args.e2e_steps is not None else min(args.steps, 5)
    Uh = torch.from_numpy(U).pin_memory()
    h2d = Uh.numel() * 16
    d2h = 6 * BLOCK * 9 * DIMS[3] * 16
    barrier()
    e0 = time.perf_counter()
    for i in range(e2e_steps):
        step(args.warmup + i, "fp16", Uh)
    barrier()
    t_e2e = max_over_ranks(time.perf_counter() - e0)
    e2e_value = job_rate(BLOCK * e2e_steps, world, t_e2e)

    # ---- roofline of the dominant kernel class of the FP16 noise phase
    dom = max(tm, key=lambda k: tm[k][0])
    ms, nl, units = tm[dom]
    roofline = {"kernel": dom, "bound": "hbm", "achieved": None, "peak": HBM_PEAK_GBS, "unit": "GB/s",
                "frac": None, "traffic": None, "peak_source": "MEASURED_PEAKS.json hbm_gbs (of measured)",
                "avg_launch_ms": ms / max(nl, 1), "launches": nl,
                "bytes_per_launch": tbytes.get(dom, 0.0) / max(nl, 1),
                "breakdown_ms": {k: round(v[0], 2) for k, v in tm.items() if v[0] > 0},
                "breakdown_launches": {k: v[1] for k, v in tm.items() if v[1] > 0},
                "class_gbs": {k: round(tbytes[k] / (v[0] / 1000.0) / 1e9, 1) for k, v in tm.items()
                              if v[0] > 0 and tbytes.get(k, 0) > 0}}
    if tbytes.get(dom, 0) > 0 and ms > 0:
        roofline["achieved"] = tbytes[dom] / (ms / 1000.0) / 1e9
        roofline["frac"] = roofline["achieved"] / HBM_PEAK_GBS
        if dom in DRAM_PER_ALGORITHMIC:
            # DRAM bytes per launch: the ratio ncu measured on the same kernels (smaller lattice, the
            # bytes per launch in proportion to the vectors read) times this run's algorithmic bytes
            ratio, src = DRAM_PER_ALGORITHMIC[dom]
            roofline["traffic"] = ratio * roofline["bytes_per_launch"]
            roofline["traffic_source"] = src

    info_lam_min = lam_min
    loop.close()
    ctx.close()
    del Ud
    torch.cuda.empty_cache()
    cfg2 = None if args.no_cfg2 else cfg2_fp64(torch)
    cfg3 = cfg5 = None
    if not args.no_cfg35:
        for name, fn in (("cfg3", cfg3_batching), ("cfg5", cfg5_derivs)):
            try:
                r = fn(torch)
            except Exception as e:  # reported, not fatal: the headline numbers above stand on their own
                r = {"error": str(e)[:300]}
            torch.cuda.empty_cache()
            if name == "cfg3":
                cfg3 = r
            else:
                cfg5 = r
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
        one = oracle_sample_threads(1)
        cpu["one_thread"] = None if one is None else {"value": one[0], "unit": "estimates/s", "cores": 1,
                                                     "sample_s": one[1],
                                                     "how": "the same sample in a child process with its "
                                                            "BLAS / OpenMP thread pools set to 1"}

    if rank == 0:
        line = {"metric": "deflated loop estimates/s at 1e-10 true residual", "value": value, "unit": "estimates/s",
                "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
                "ms_per_step": 1000.0 * t_max / args.steps, "higher_is_better": True, "scaling": "weak",
                "vs_baseline": None, "dtype": "f32", "data": "synthetic",
                "config": {"workload": WORKLOAD, "lattice": "24x24x24x32", "kappa": KAPPA, "noises": NNOISE,
                           "noises_per_step": BLOCK, "Q": info["Q"], "link_eps": LINK_EPS,
                           "poly_preconditioner_degree": args.prec_degree,
                           "precision": "FP16 storage of the inner Krylov basis, FP32 arithmetic, FP64 outer "
                                        "true residual, FP64 setup; HFES projections split-precision FP64 on "
                                        "tensor cores",
                           "inner_tol": INNER_TOL, "inner_gram_schmidt_passes": 1, "inner_m": HEAD_M_INNER,
                           "inner_lanczos_window": INNER_WINDOW,
                           "l2": "inputs larger than L2 (Krylov bases of 10 noises: GBs per step)",
                           "parallelism": "independent gauge configuration per rank" if world > 1 else "single GPU"},
                "gpu_launches": launches,
                "setup_s": setup_s, "setup_matvecs": info["matvecs_setup"], "eig_resid_max": info["eig_resid_max"],
                "amortised_estimates_per_s": NNOISE / (setup_s + NNOISE * per_noise_s),
                "matvecs_per_noise": float(np.mean([s["matvecs"] for s in stats]) / BLOCK),
                "max_true_resid": max(s["max_true_resid"] for s in stats),
                "roofline": roofline,
                "e2e": {"value": e2e_value, "unit": "estimates/s", "h2d_bytes_per_step": int(h2d),
                        "d2h_bytes_per_step": int(d2h), "steps": e2e_steps},
                "clocks": clk, "cpu_baseline": cpu,
                "bf16": {"value": BLOCK * nb16 * world / t_bf16, "unit": "estimates/s", "steps": nb16},
                "fp64_plain": {"value": BLOCK * world / t_fp64, "unit": "estimates/s", "steps": 1,
                               "speedup_fp16_vs_fp64": value / (BLOCK * world / t_fp64),
                               "speedup_bf16_vs_fp64": (BLOCK * nb16 / t_bf16) / (BLOCK / t_fp64)},
                "estimate_vs_fp64": errors,
                "cfg2_fp64": cfg2, "cfg3_16x32_fp64": cfg3, "cfg5_derivs": cfg5, "dslash": dslash, "deflation_tensor_cores": deflation, "batching": batching}
        print(json.dumps(line))
    if world > 1:
        torch.distributed.destroy_process_group()


if __name__ == "__main__":
    main()
