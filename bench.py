"""Benchmark of the batched IESH step on GB300.

Workload (default): harmonic double-well Newns-Anderson model, M=100 bath
states (N=101 orbitals), Ne=50 electrons, 4096 trajectories with thermal
initial conditions at kT in {0.005, 0.0075, 0.01}, dt=1 a.u., FP64 path.
A step is one pass of the whole IESH step (eigenpairs, force, couplings,
exponential integrator, determinant-ratio hop probabilities, hop and
rescale) over the whole batch.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

Prints one JSON line.  --impl reference times the FP64 CPU oracle on the
host cores on a bounded sample of the same workload.
"""
import argparse
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import iesh_inputs as W  # noqa: E402

METRIC = "IESH trajectory-steps/s (batched, 1 GB300) vs plain FP64 path; % of roofline"
UNIT = "traj-steps/s"
MEASURED_PEAKS = os.path.join(ROOT, "MEASURED_PEAKS.json")
# FP64 peak derived from the unit counts and clocks: 2 DFMA per clock per SM
# (ncu's dfma peak counter), 152 SMs, 2.07 GHz maximum SM clock
FP64_NOMINAL_TFLOPS = 2 * 2 * 152 * 2.07e9 / 1e12
FP32_NOMINAL_TFLOPS = 152 * 128 * 2 * 2.07e9 / 1e12  # FP32 SIMT at the maximum SM clock
TF32_PER_BF16 = 1.1 / 2.25  # nominal dense TF32 : BF16 tensor rate
# DRAM bytes (read + write) per trajectory of one launch of the dominant kernel, by
# (kernel, N, Ne), from ncu captures (dram__bytes_read.sum + dram__bytes_write.sum) of
# the named batch size, divided by it: the traffic is per-trajectory streams of C and
# W, so it scales with the batch.  A shape or kernel not in the table reports null.
DRAM_BYTES_PER_TRAJ = {
    # k_cheb, dram__bytes_read.sum + dram__bytes_write.sum of a
    # 1024-trajectory capture / 1024
    ("k_cheb", 101, 50): (170.948096e6 + 47.242752e6) / 1024,
    ("k_cheb", 201, 100): (675.789824e6 + 293.651456e6) / 1024,
}


def measured_peaks():
    try:
        with open(MEASURED_PEAKS) as f:
            return json.load(f)
    except (OSError, ValueError):
        return {}


def workload(M=100, n_traj=4096, dt=1.0):
    md = W.double_well(M)
    kT = np.array([0.005, 0.0075, 0.01])[np.arange(n_traj) % 3]
    return md, kT, dt


def initial_state(md, kT, n, seed):
    x, p = W.thermal_harmonic(n, md["mass"], md["par"][0], kT, seed)
    occ = W.lowest_occupations(n, md["Ne"])
    C = W.unit_coefficients(occ, md["M"] + 1)
    return x, p, occ, C


# --------------------------------------------------------------- clocks
class ClockSampler:
    QUERY = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.path = None

    def __enter__(self):
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.QUERY}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except OSError:
            self.proc = None
        time.sleep(0.3)
        return self

    def __exit__(self, *a):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self):
        rows = []
        try:
            for line in open(self.path):
                f = [v.strip() for v in line.split(",")]
                if len(f) >= 9:
                    rows.append(f)
        finally:
            try:
                os.unlink(self.path)
            except OSError:
                pass
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unavailable"], "samples": 0}

        def num(v):
            try:
                return float(v)
            except ValueError:
                return None

        sm = [num(r[1]) for r in rows if num(r[1]) is not None]
        mx = [num(r[2]) for r in rows if num(r[2]) is not None]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in rows for i in range(4)
                          if r[5 + i].lower() in ("active", "0x1", "1")})
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(mx) if mx else None, "reasons": reasons,
                "samples": len(rows)}


# ------------------------------------------------------------- replicas
def replica_traj_base(rank, n_per_rank):
    """Global id of a replica's first trajectory.  Every rank uses the same
    Philox key; its trajectories draw with global ids rank * n_per_rank + t,
    so an N-GPU job computes the same trajectories as one GPU holding the
    whole batch."""
    return rank * n_per_rank


def replica_slice(rank, n_per_rank):
    """The rank's trajectories within the whole job's batch."""
    return slice(rank * n_per_rank, (rank + 1) * n_per_rank)


def replica_state(M, n, world, rank, dt=1.0):
    """The rank's slice of the whole job's seeded initial state (the batch of
    n * world trajectories that one GPU would run)."""
    md, kT, dt = workload(M, n * world, dt)
    x, p, occ, C = initial_state(md, kT, n * world, seed=1000)
    sl = replica_slice(rank, n)
    return md, dt, x[sl].copy(), p[sl].copy(), occ[sl].copy(), C[sl].copy()


def aggregate(ms_local, e2e_local, n_per_rank, steps, world, dist=None, device="cpu"):
    """Whole-job throughput of independent replicas: the slowest rank's time
    bounds the job (max over ranks), the units are summed over ranks."""
    ms, e2e = ms_local, e2e_local
    if dist is not None and world > 1:
        import torch
        t = torch.tensor([ms_local, e2e_local], dtype=torch.float64, device=device)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        ms, e2e = float(t[0]), float(t[1])
    value = world * n_per_rank * steps / (ms / 1e3) if ms > 0 else None
    return dict(ms=ms, e2e_s=e2e, value=value)


# ------------------------------------------------------------- our arm
def useful_flops(N, Ne):
    """Algorithmic work of one trajectory-step (flops): unitary application
    8 N^2 Ne, ratio GEMM 8 (N - Ne) Ne^2, overlap LU (8/3) Ne^3, warm-started
    secular eigensolver about 8 x 3 N^2, coupling generation about 10 N^2."""
    prop = 8.0 * N * N * Ne
    step = prop + 8.0 * (N - Ne) * Ne * Ne + 8.0 / 3.0 * Ne ** 3 + 24.0 * N * N + 10.0 * N * N
    return prop, step


def tf32_peak():
    bf16 = measured_peaks().get("bf16_tflops")
    if bf16:
        return bf16 * TF32_PER_BF16, ("of measured: MEASURED_PEAKS.json bf16_tflops x nominal "
                                      "TF32/BF16 ratio 1.1/2.25")
    return 1900.0 * TF32_PER_BF16, "of fallback: 1.9 PFLOP/s bf16 x 1.1/2.25"


def run_ours(args):
    import torch
    import torch.distributed as dist

    import paper_2212_00518_gb300 as P
    from paper_2212_00518_gb300 import build as B

    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    if world > 1:
        dist.init_process_group("nccl")
    if rank == 0 or world > 1:
        B.build()
    if world > 1:
        dist.barrier()
    stream = torch.cuda.current_stream()
    seed = args.seed

    def barrier():
        if world > 1:
            dist.barrier()
        torch.cuda.synchronize()

    def agg(ms=0.0, sec=0.0):
        a = aggregate(ms, sec, 1, 1, world, dist if world > 1 else None, "cuda")
        return a["ms"], a["e2e_s"]

    def config_state(M, n):
        return replica_state(M, n, world, rank, args.dt)

    def measure(md, dt, x, p, occ, C, precision, sample_clocks=False, propagator=0, e2e=True):
        n = x.shape[0]
        c = P.Context(md, n, precision=precision, stream=stream.cuda_stream, propagator=propagator,
                      skip_bound=args.skip_bound, traj_base=replica_traj_base(rank, n),
                      deflation=not args.no_deflation)
        c.set_state(x, p, occ, C if precision == P.PREC_FP64 else C.astype(np.complex64))
        for _ in range(args.warmup):
            c.run(dt, 1, seed)
        torch.cuda.synchronize()
        ev0 = torch.cuda.Event(enable_timing=True)
        ev1 = torch.cuda.Event(enable_timing=True)
        c.profile(True)
        barrier()
        clk = ClockSampler(local) if sample_clocks else None
        if clk:
            clk.__enter__()
        ev0.record(stream)
        for _ in range(args.steps):
            c.run(dt, 1, seed)
        ev1.record(stream)
        barrier()
        if clk:
            clk.__exit__()
        ms, _ = agg(ms=ev0.elapsed_time(ev1))
        prof = c.profile_read()
        c.profile(False)
        shape = c.kernel_shape()[0]
        out = dict(ms=ms, prof=prof, K=c.propagator_terms(), tc=shape if shape in (8, 16) else 0,
                   status=c.get_state()["status"], clocks=clk.summary() if clk else None, n=n)
        if e2e:
            # end to end through the C-ABI: every step takes the whole state from a
            # pinned host checkpoint and writes the advanced state back to it
            # (iesh_run_host: copies in and out overlapped with the step over
            # trajectory ranges)
            blob = torch.from_numpy(c.checkpoint_save()).pin_memory()
            steps = max(1, min(args.steps, args.e2e_steps))
            barrier()
            t0 = time.perf_counter()
            for _ in range(steps):
                c.run_host(blob, blob, dt, 1, seed, chunks=args.e2e_chunks)
            barrier()
            _, sec = agg(sec=time.perf_counter() - t0)
            out["e2e"] = {"value": world * n * steps / sec, "unit": UNIT,
                          "h2d_bytes_per_step": int(blob.numel()),
                          "d2h_bytes_per_step": int(blob.numel()),
                          "steps": steps,
                          "chunks": args.e2e_chunks,
                          "what": "per step: iesh_run_host of the whole trajectory state held in "
                                  "pinned host memory (the checkpoint of bit-exact resume): copied "
                                  "in, advanced one step and copied back, over trajectory ranges "
                                  "whose copies overlap the other ranges' step"}
        c.close()
        return out

    def shares(prof):
        tot = max(1e-9, sum(u[0] for u in prof.values()))
        return {k: round(v[0] / tot, 4) for k, v in prof.items() if v[1]}

    def fp64_roofline(r, N, Ne):
        """The FP64 propagator k_cheb against the derived FP64 peak: useful work
        8 N^2 Ne per trajectory-step (achieved, frac) and executed work K 4 N^2 Ne
        (executed_*, the FP64 pipe's utilisation)."""
        n = r["n"]
        pm, pn = r["prof"]["propagate"]
        t = pm / pn / 1e3 if pn else None
        prop_w, step_w = useful_flops(N, Ne)
        ach = prop_w * n / t / 1e12 if t else None
        exe = float(np.sum(r["K"].astype(np.float64))) * 4.0 * N * N * Ne / t / 1e12 if t else None
        tr = DRAM_BYTES_PER_TRAJ.get(("k_cheb", N, Ne))
        step_s = r["ms"] / args.steps / 1e3
        return {"bound": "alu", "kernel": "k_cheb (Chebyshev exponential integrator, FP64)",
                "achieved": ach, "peak": FP64_NOMINAL_TFLOPS, "unit": "TFLOP/s",
                "frac": ach / FP64_NOMINAL_TFLOPS if ach else None,
                "achieved_is": "algorithmic 8 N^2 Ne flops per trajectory-step (unitary "
                               "application) x trajectories / mean k_cheb launch time",
                "executed_achieved": exe,
                "executed_frac": exe / FP64_NOMINAL_TFLOPS if exe else None,
                "executed_is": "K 4 N^2 Ne flops actually issued (K Chebyshev orders of a "
                               "real N x N by complex N x Ne product; K over the bulk interval where "
                               "the isolated top level is deflated)",
                "mean_cheb_terms": float(r["K"].mean()),
                "peak_source": "derived: 2 DFMA/clk/SM x 152 SMs x 2.07 GHz (no measured FP64 "
                               "peak in MEASURED_PEAKS.json; a DFMA probe measured 1.20)",
                "traffic": tr * n if tr else None,
                "traffic_source": "ncu dram__bytes_read.sum + dram__bytes_write.sum per "
                                  "trajectory of a capture at this shape, times the batch"
                                  if tr else "no capture at this shape",
                "step_useful_tflops": step_w * n / step_s / 1e12,
                "step_useful_frac": step_w * n / step_s / 1e12 / FP64_NOMINAL_TFLOPS,
                "kernel_time_share": shares(r["prof"])}

    def mixed_roofline(r, N, Ne):
        n = r["n"]
        pm, pn = r["prof"]["propagate"]
        t = pm / pn / 1e3 if pn else None
        prop_w, step_w = useful_flops(N, Ne)
        ach = prop_w * n / t / 1e12 if t else None
        exe = float(np.sum(r["K"].astype(np.float64))) * 4.0 * N * N * Ne / t / 1e12 if t else None
        ptf, src = tf32_peak()
        step_s = r["ms"] / args.steps / 1e3
        # time bound of the whole step: FP32/TF32 contractions on the tensor cores,
        # eigen and coupling generation on the FP64 pipe
        w_tc = prop_w + 8.0 * (N - Ne) * Ne * Ne + 8.0 / 3.0 * Ne ** 3
        w_64 = step_w - w_tc
        t_star = w_tc / (ptf * 1e12) + w_64 / (FP64_NOMINAL_TFLOPS * 1e12)
        if r["tc"] == 16:
            # FP16 operands: the dense FP16 rate equals the bf16 one
            Kp, NB = (N + 15) // 16 * 16, (2 * Ne + 15) // 16 * 16
            pbf = measured_peaks().get("bf16_tflops")
            roof = {"bound": "tensor", "kernel": "k_cheb_tc16 (tcgen05 kind::f16, FP16 split operands, "
                                                 "two CTAs per SM)",
                    "peak": pbf if pbf else 1900.0,
                    "peak_source": ("of measured: MEASURED_PEAKS.json bf16_tflops (FP16 dense = bf16 dense)"
                                    if pbf else "of fallback: 1.9 PFLOP/s bf16 burst"),
                    "executed_tensor_tflops": exe * 3 * (128 * Kp * NB) / (N * N * 2 * Ne) if exe else None}
        elif r["tc"]:
            Kp, NB = (N + 7) // 8 * 8, (2 * Ne + 15) // 16 * 16
            roof = {"bound": "tensor", "kernel": "k_cheb_tc (tcgen05 kind::tf32, 3xTF32)",
                    "peak": ptf, "peak_source": src,
                    "executed_tensor_tflops": exe * 3 * (128 * Kp * NB) / (N * N * 2 * Ne) if exe else None}
        else:
            roof = {"bound": "alu", "kernel": "k_cheb_f32t (register-tiled FP32 SIMT)",
                    "peak": FP32_NOMINAL_TFLOPS,
                    "peak_source": "nominal FP32 SIMT (152 SMs x 128 FMA x 2 x 2.07 GHz)",
                    "tf32_tensor_frac": ach / ptf if ach else None}
        roof.update({"achieved": ach, "unit": "TFLOP/s",
                     "frac": ach / roof["peak"] if ach else None,
                     "achieved_is": "algorithmic 8 N^2 Ne flops per trajectory-step x "
                                    "trajectories / mean propagator launch time",
                     "executed_fp32_tflops": exe, "mean_cheb_terms": float(r["K"].mean()),
                     "step_roofline_time_frac": n * t_star / step_s,
                     "step_roofline_is": "t* = (8N^2Ne + 8(N-Ne)Ne^2 + 8/3 Ne^3) / P_TF32 + "
                                         "(24 N^2 + 10 N^2) / P_FP64 per trajectory-step, "
                                         "divided by the measured time per trajectory-step"})
        return roof

    MIXED_DTYPE = ("f32 coefficients, coupling generator, propagation (tensor cores for N <= 128: "
                   "FP16 hi + lo split operands, about 22 bits each, FP32 accumulation, where two CTAs "
                   "fit an SM, else 3xTF32; FP32 SIMT above), overlap LU or Gauss-Jordan ratios; "
                   "double-float secular sums; f64 eigen iteration, forces, hop selection and rescale")

    # ---------------------------------------------- headline: M = args.M
    n = args.n_traj
    md, dt, x, p, occ, C = config_state(args.M, n)
    N, Ne = md["M"] + 1, md["Ne"]
    r64 = measure(md, dt, x, p, occ, C, P.PREC_FP64, sample_clocks=True)
    rmx = None if args.no_mixed else measure(md, dt, x, p, occ, C, P.PREC_MIXED)
    rov = None if args.no_overlap else measure(md, dt, x, p, occ, C, P.PREC_FP64,
                                               propagator=P.iesh.PROP_OVERLAP, e2e=False)
    # ---------------------------------------------- config 3: M = 200, Ne = 100
    c3 = None
    if not args.no_config3 and args.M != 200:
        n3 = args.c3_traj
        md3, dt3, x3, p3, occ3, C3 = config_state(200, n3)
        c3_64 = measure(md3, dt3, x3, p3, occ3, C3, P.PREC_FP64, sample_clocks=True)
        c3_mx = measure(md3, dt3, x3, p3, occ3, C3, P.PREC_MIXED, sample_clocks=True)
        c3 = (md3, dt3, n3, c3_64, c3_mx)

    if rank == 0:
        value = world * n * args.steps / (r64["ms"] / 1e3)
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": r64["ms"] / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic",
            "config": {"workload": f"double-well Newns-Anderson IESH, M={args.M} bath states, "
                                   f"Ne={Ne}, {n} trajectories per GPU, kT 0.005-0.01, "
                                   f"dt={dt} a.u., FP64 path",
                       "trajectories_per_gpu": n, "n_orbitals": N, "n_electrons": Ne,
                       "precision": "fp64", "skip_bound": bool(args.skip_bound),
                       "l2": "working set > L2 (coefficients + coupling matrices "
                             f"{(n * Ne * N * 16 + n * N * N * 8) / 1e9:.2f} GB)",
                       "replicas": "rank r holds global trajectories [r n, (r+1) n) of one "
                                   "seeded batch, Philox ids = global ids",
                       "status_nonzero": int(np.count_nonzero(r64["status"]))},
            "roofline": fp64_roofline(r64, N, Ne),
            "e2e": r64["e2e"],
            "gpu_launches": int(sum(v[1] for v in r64["prof"].values())),
            "clocks": r64["clocks"],
            "impl": "ours",
        }
        if rmx is not None:
            line["mixed"] = {
                "value": world * n * args.steps / (rmx["ms"] / 1e3), "unit": UNIT,
                "ms_per_step": rmx["ms"] / args.steps, "speedup_vs_fp64": r64["ms"] / rmx["ms"],
                "dtype": MIXED_DTYPE, "kernel_time_share": shares(rmx["prof"]),
                "roofline_propagate": mixed_roofline(rmx, N, Ne), "e2e": rmx["e2e"],
                "gpu_launches": int(sum(v[1] for v in rmx["prof"].values())),
                "status_nonzero": int(np.count_nonzero(rmx["status"])),
            }
        if rov is not None:
            po_ms, po_n = rov["prof"]["propagate"]
            ach_o = 4.0 * N * N * Ne * n / (po_ms / po_n / 1e3) / 1e12 if po_n else None
            line["overlap"] = {
                "value": world * n * args.steps / (rov["ms"] / 1e3), "unit": UNIT,
                "ms_per_step": rov["ms"] / args.steps, "speedup_vs_fp64": r64["ms"] / rov["ms"],
                "dtype": "f64",
                "propagator": "diabatic-basis variant: exp(-i L1 dt/2) Q1^T Q0 exp(-i L0 dt/2), "
                              "O from the arrowhead's closed form (second order, like the "
                              "averaged generator)",
                "kernel_time_share": shares(rov["prof"]),
                "propagate_tflops": ach_o,
                "gpu_launches": int(sum(v[1] for v in rov["prof"].values())),
                "status_nonzero": int(np.count_nonzero(rov["status"])),
            }
        if c3 is not None:
            md3, dt3, n3, a, b = c3
            N3, Ne3 = md3["M"] + 1, md3["Ne"]
            line["config3"] = {
                "workload": f"double-well Newns-Anderson IESH, M=200 bath states, Ne={Ne3}, "
                            f"{n3} trajectories per GPU, kT 0.005-0.01, dt={dt3} a.u.",
                "fp64": {"value": world * n3 * args.steps / (a["ms"] / 1e3), "unit": UNIT,
                         "ms_per_step": a["ms"] / args.steps, "dtype": "f64",
                         "roofline": fp64_roofline(a, N3, Ne3), "e2e": a["e2e"],
                         "clocks": a["clocks"],
                         "status_nonzero": int(np.count_nonzero(a["status"]))},
                "mixed": {"value": world * n3 * args.steps / (b["ms"] / 1e3), "unit": UNIT,
                          "ms_per_step": b["ms"] / args.steps, "dtype": MIXED_DTYPE,
                          "kernel_time_share": shares(b["prof"]),
                          "roofline_propagate": mixed_roofline(b, N3, Ne3), "e2e": b["e2e"],
                          "clocks": b["clocks"],
                          "status_nonzero": int(np.count_nonzero(b["status"]))},
                "speedup_mixed_vs_fp64": a["ms"] / b["ms"],
            }
        if world == 1 and not args.no_cpu_baseline:
            md0, kT0, _ = workload(args.M, n, args.dt)
            line["cpu_baseline"] = cpu_baseline(args, md0, kT0, dt)
        print(json.dumps(line), flush=True)
    if world > 1:
        dist.destroy_process_group()


# -------------------------------------------------------- CPU oracle arm
def _oracle_sample(md, kT, dt, n_traj, n_steps, seed, threads):
    from oracle import oracle as O
    B = O.bind(md)
    x, p, occ, C = initial_state(md, kT[:n_traj], n_traj, seed=1000)
    t0 = time.perf_counter()
    O.run(B, x, p, occ.astype(np.int32), np.transpose(C, (0, 2, 1)), dt, n_steps, seed,
          n_threads=threads)
    return time.perf_counter() - t0


def cpu_baseline(args, md, kT, dt):
    cores = os.cpu_count() or 1
    n_traj = 2 * cores
    steps = args.cpu_steps
    sec = _oracle_sample(md, kT, dt, n_traj, steps, args.seed, cores)
    return {"value": n_traj * steps / sec, "unit": UNIT, "cores": cores, "kind": "oracle",
            "sample": f"{n_traj} trajectories x {steps} steps of the same workload "
                      f"({sec:.1f} s, one trajectory per thread)"}


def run_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    md, kT, dt = workload(args.M, args.n_traj, args.dt)
    cores = os.cpu_count() or 1
    n_traj = 2 * cores
    per_step = []
    for _ in range(args.warmup):
        _oracle_sample(md, kT, dt, n_traj, 1, args.seed, cores)
    for _ in range(args.steps):
        per_step.append(_oracle_sample(md, kT, dt, n_traj, 1, args.seed, cores))
    sec = sum(per_step)
    value = n_traj * args.steps / sec
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": 1, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": 1e3 * sec / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": f"double-well Newns-Anderson IESH, M={args.M} bath states, "
                               f"Ne={md['Ne']}, bounded sample of {n_traj} trajectories per "
                               f"step, dt={dt} a.u., FP64 CPU oracle"},
        "impl": "reference",
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle",
                         "sample": f"{n_traj} trajectories x 1 step per timed step"},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


# ------------------------------------------------------ other workloads
def _timed_steps(torch, stream, fn, warmup, steps):
    for _ in range(warmup):
        fn()
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(steps):
        fn()
    e1.record(stream)
    torch.cuda.synchronize()
    return e0.elapsed_time(e1)


def run_workload(args):
    """Secondary measurements (one JSON line each): the paper-shaped timing
    grid, the uneven scattering batch, the desorption/scattering ensembles of
    the desorption model, E_occ."""
    import torch

    import paper_2212_00518_gb300 as P
    from paper_2212_00518_gb300 import build as B
    B.build()
    stream = torch.cuda.current_stream()
    line = {"unit": UNIT, "n_gpus": 1, "steps": args.steps, "warmup": args.warmup,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "data": "synthetic",
            "impl": "ours"}
    if args.workload == "paper":
        # Sec. III B double well with the paper's constants, dt = 10 a.u.
        res = []
        for M in (40, 80, 200):
            md = W.double_well_paper(M)
            for n in (1, 4096):
                x, p = W.thermal_harmonic(n, md["mass"], md["par"][0], 5 * 9.5e-4, seed=1)
                occ = W.lowest_occupations(n, md["Ne"])
                C = W.unit_coefficients(occ, M + 1)
                for prec in (P.PREC_FP64, P.PREC_MIXED):
                    for skip in (False, True):
                        c = P.Context(md, n, precision=prec, skip_bound=skip, stream=stream.cuda_stream)
                        c.set_state(x, p, occ, C if prec == P.PREC_FP64 else C.astype(np.complex64))
                        ms = _timed_steps(torch, stream, lambda: c.run(10.0, 1, 0), args.warmup, args.steps)
                        _, hops, _ = c.counters()
                        res.append({"M": M, "trajectories": n, "precision": "fp64" if prec == 0 else "mixed",
                                    "skip_bound": skip, "traj_steps_per_s": n * args.steps / (ms / 1e3),
                                    "ms_per_step": ms / args.steps, "hops": int(hops.sum())})
                        c.close()
        pick = [r for r in res if r["M"] == 80 and r["trajectories"] == 4096
                and r["precision"] == "fp64" and not r["skip_bound"]][0]
        line.update(metric=METRIC + " [paper double well, Sec. III B constants, dt=10]",
                    value=pick["traj_steps_per_s"], dtype="f64",
                    config={"workload": "paper-shaped timing grid: M in {40, 80, 200}, 1 and 4096 "
                                        "trajectories, FP64 and mixed, with and without the "
                                        "hop-probability bound skip", "value_is": "M=80, 4096, fp64, no skip"},
                    results=res)
    elif args.workload == "scatter":
        # the uneven batch run to completion: every trajectory until it leaves
        # the surface (z > 10 angstrom) or 300 fs, all nine (M, bias) contexts
        # in one device-side loop (one graph launch), live steps counted exactly
        from paper_2212_00518_gb300.ensemble import UnevenBatch
        groups = W.scattering_batch(16384, seed=4)
        dt, chunk = 0.1 * W.FS_AU, 64
        cap = int(round(300.0 * W.FS_AU / dt))
        warm = UnevenBatch(groups, dt=dt, z_done=W.angstrom(10.0), precision=P.PREC_MIXED,
                           compact_every=chunk, seed=0, autotune=args.autotune)
        warm.run(chunk * max(3, args.warmup))
        warm.close()
        ub = UnevenBatch(groups, dt=dt, z_done=W.angstrom(10.0), precision=P.PREC_MIXED,
                         compact_every=chunk, seed=0, autotune=args.autotune)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        with ClockSampler(0) as clk:
            e0.record(ub.stream)
            live_steps = ub.run(cap)
            e1.record(ub.stream)
            torch.cuda.synchronize()
        sec = e0.elapsed_time(e1) / 1e3
        res = ub.results()
        loop_steps, live_left = ub.ens.status()
        n_total = int(sum(len(g["x"]) for g in groups))
        kernels_per_step = 5  # eigen, coupling, propagation, hop, norm check
        launches = (loop_steps // chunk) * (len(groups) * (chunk * kernels_per_step + 1) + 1)
        done = (res["status"] & P.iesh.TRAJ_DONE) != 0
        line.update(metric=METRIC + " [uneven scattering batch, run to completion]",
                    value=live_steps / sec, steps=int(loop_steps), warmup=chunk * max(3, args.warmup),
                    ms_per_step=1e3 * sec / max(1, loop_steps),
                    dtype="mixed (f32 coupling, propagation, LU and ratio solves; double-float secular sums; "
                          "f64 eigen iteration, forces, rescale)",
                    config={"workload": "16384 Morse + image-charge scattering trajectories, M in "
                                        "{50, 100, 200} (Ne = M/2), bias 0 / 0.05 / 0.1 a.u. (two "
                                        "leads), E_inc 0.2-1.5 eV from 5 angstrom, dt 0.1 fs, "
                                        "until z > 10 angstrom or 300 fs; nine contexts advanced by "
                                        "one device-side graph loop (conditional while node), work "
                                        "lists compacted on the device every 64 steps",
                            "contexts": len(groups), "trajectories": n_total,
                            "live_traj_steps": int(live_steps),
                            "value_is": "live trajectory-steps (sum of the trajectories' own step "
                                        "counters) / CUDA-event time of the single graph launch",
                            "graph_launches": 1, "loop_steps": int(loop_steps),
                            "finished": int(done.sum()), "live_at_end": int(live_left),
                            "mean_steps_per_trajectory": float(res["nstep"].mean())},
                    gpu_launches=int(launches), clocks=clk.summary())
        ub.close()
    elif args.workload == "erpenbeck":
        # Sec. III C desorption and Sec. III D scattering on the desorption model
        # with the paper's converged settings: 100 GL states, band 64 eV,
        # Gamma = 1 eV, dt = 0.1 fs, threshold 5 angstrom; mixed precision.
        dt = 0.1 * W.FS_AU
        thr = W.angstrom(5.0)
        kT = 300 * W.KB_HARTREE_PER_K
        md = W.desorption(1.0, 100, band_ev=64.0)
        warm = P.Context(md, 64, precision=P.PREC_MIXED, stream=stream.cuda_stream)
        warm.init_state(64, kT_nuc=kT, kT_el=kT, seed=99)
        warm.run(dt, max(1, args.warmup), 0)
        warm.close()

        def timed_run(ctx, n_steps):
            ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            torch.cuda.synchronize()
            ev0.record(stream)
            ctx.run(dt, n_steps, 1)
            ev1.record(stream)
            torch.cuda.synchronize()
            return ev0.elapsed_time(ev1) / 1e3

        n_des, steps_des = 2048, 2000  # 200 fs
        c = P.Context(md, n_des, precision=P.PREC_MIXED, z_done=thr, compact_every=64,
                      stream=stream.cuda_stream)
        c.init_state(n_des, kT_nuc=kT, kT_el=kT, seed=1)
        sec = timed_run(c, steps_des)
        st = c.get_state()
        ns = c.counters()[0]
        done = (st["status"] & P.iesh.TRAJ_DONE) != 0
        pdes = {f"{t} fs": float(np.mean(done & (ns <= int(round(t * W.FS_AU / dt)))))
                for t in (50, 100, 150, 200)}
        des = {"trajectories": n_des, "steps": steps_des, "live_traj_steps": int(ns.sum()),
               "live_traj_steps_per_s": float(ns.sum()) / sec, "seconds": sec, "P_des": pdes}
        c.close()
        scat = []
        for E in (0.25, 0.5, 1.0, 1.5):
            n_sc = 1024
            mds, x, p, occ, C = W.erpenbeck_scattering(n_sc, E, M=100, band_ev=64.0)
            c = P.Context(mds, n_sc, precision=P.PREC_MIXED, z_done=thr, compact_every=64,
                          stream=stream.cuda_stream)
            c.set_state(x, p, occ, C.astype(np.complex64))
            sec = timed_run(c, 3000)  # 300 fs
            st = c.get_state()
            ns = c.counters()[0]
            done = (st["status"] & P.iesh.TRAJ_DONE) != 0
            loss = W.ev(E) - st["p"][done] ** 2 / (2 * mds["mass"])
            scat.append({"E_inc_eV": E, "rebounded": float(done.mean()),
                         "KE_loss_eV": float(loss.mean() / W.ev(1.0)) if done.any() else None,
                         "KE_loss_se_eV": float(loss.std() / np.sqrt(max(done.sum(), 1)) / W.ev(1.0)),
                         "live_traj_steps_per_s": float(ns.sum()) / sec})
            c.close()
        line.update(metric=METRIC + " [desorption model: Sec. III C desorption, Sec. III D scattering]",
                    value=des["live_traj_steps_per_s"],
                    dtype="mixed (f32 coupling, propagation, LU and ratio solves; double-float "
                          "secular sums; f64 eigen iteration, forces, rescale)",
                    config={"workload": "desorption model (Table II), 100 GL states, band 64 eV, "
                                        "Gamma 1 eV, dt 0.1 fs, threshold 5 angstrom, work list "
                                        "compacted every 64 steps; desorption: 2048 trajectories, "
                                        "Wigner 300 K nuclei and canonical 300 K electrons, 200 fs; "
                                        "scattering: 1024 trajectories per E_inc from 5 angstrom, "
                                        "0 K electrons, up to 300 fs",
                            "value_is": "desorption live trajectory-steps/s"},
                    results={"desorption": des, "scattering": scat})
    elif args.workload == "relaxation":
        # Sec. III B double-well relaxation: 40 bath states, band 10 Gamma,
        # 1000 trajectories from Boltzmann nuclei at 5 kT and canonical
        # electrons at kT, dt = 100 a.u., 10^5 steps (10^7 a.u.); 1 - P_d
        # (hole-impurity population) and the mean kinetic energy every 1000
        # steps, GL and trapezoid baths.
        kT, dt, n, chunks, every = 9.5e-4, 100.0, 1000, 100, 1000
        res = {}
        total_steps, total_sec = 0, 0.0
        for disc in ("gl", "trapezoid"):
            md = W.double_well_paper(40, disc=disc)
            c = P.Context(md, n, precision=P.PREC_MIXED, stream=stream.cuda_stream)
            c.init_state(n, kT_nuc=5 * kT, kT_el=kT, seed=7)
            hole, ke = [], []
            torch.cuda.synchronize()
            for _ in range(chunks):
                ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                ev0.record(stream)
                c.run(dt, every, 0)
                ev1.record(stream)
                st = c.get_state()  # synchronises
                total_sec += ev0.elapsed_time(ev1) / 1e3
                total_steps += n * every
                lam, q0, _ = c.eigen()
                # wavefunction impurity population sum_e |sum_i q0_i C_ie|^2
                amp = np.einsum("ti,tei->te", q0, st["C"])
                hole.append(float(1.0 - np.mean(np.sum(np.abs(amp) ** 2, axis=1))))
                ke.append(float(np.mean(st["p"] ** 2) / (2 * md["mass"])))
            res[disc] = {"t_au": [dt * every * (k + 1) for k in range(chunks)], "hole_population": hole,
                         "kinetic_energy": ke, "KE_over_kT_final": ke[-1] / kT}
            c.close()
        line.update(metric=METRIC + " [double-well relaxation, Sec. III B]", value=total_steps / total_sec,
                    dtype="mixed (f32 coupling, propagation, LU and ratio solves; double-float "
                          "secular sums; f64 eigen iteration, forces, rescale)",
                    config={"workload": "paper double well (m=2000, w=2e-4, g=20.6097, dG=-3.8e-3, "
                                        "Gamma=6.4e-3, 40 states, band 10 Gamma), 1000 trajectories, "
                                        "Boltzmann 5 kT nuclei, canonical kT electrons, dt=100, "
                                        "10^5 steps, GL and trapezoid discretisations",
                            "classical_KE_limit": kT / 2},
                    results=res)
    elif args.workload == "two":
        # Two adsorbate orbitals over six coordinates: 100 GL bath states
        # (N = 102), Ne = 51, thermal nuclei around the restraint centres,
        # random occupations with half the coefficient weight off them.
        from paper_2212_00518_gb300 import two
        n, dt = args.n_traj, 2.0
        md = W.two_orbital(100, seed=5)
        x, p, occ, C = W.two_orbital_state(md, n, 3, kT=0.01, weight=0.5)
        res = {}
        for prec, name in ((P.PREC_FP64, "fp64"), (P.PREC_MIXED, "mixed")):
            c = two.TwoOrbitalContext(md, n, precision=prec, stream=stream.cuda_stream)
            c.set_state(x, p, occ.astype(np.int16), C if prec == P.PREC_FP64 else C.astype(np.complex64))
            c.run(dt, max(3, args.warmup), 0)
            c.profile(True)
            ms = _timed_steps(torch, stream, lambda: c.run(dt, 1, 0), 0, args.steps)
            prof = c.profile_read()
            c.profile(False)
            tot = sum(v[0] for v in prof.values())
            _, hops, frus = c.counters()
            st = c.get_state()
            c.close()
            res[name] = {"traj_steps_per_s": n * args.steps / (ms / 1e3), "ms_per_step": ms / args.steps,
                         "kernel_share": {k: v[0] / tot for k, v in prof.items() if tot > 0},
                         "hops": int(hops.sum()), "frustrated": int(frus.sum()),
                         "status_nonzero": int(np.count_nonzero(st["status"]))}
        res["mixed"]["speedup_vs_fp64"] = res["mixed"]["traj_steps_per_s"] / res["fp64"]["traj_steps_per_s"]
        # oracle on one host core: a bounded sample of the same workload
        from oracle import oracle as O
        t0 = time.perf_counter()
        ns = 16
        O.run2(md, x[:ns], p[:ns], occ[:ns], np.transpose(C[:ns], (0, 2, 1)), dt, 5, 0)
        cpu = ns * 5 / (time.perf_counter() - t0)
        line.update(metric=METRIC + " [two adsorbate orbitals, six coordinates]",
                    value=res["fp64"]["traj_steps_per_s"], dtype="f64",
                    config={"workload": "two-orbital adsorbate, 100 GL bath states (N=102), Ne=51, "
                                        f"six coordinates, {n} trajectories, dt=2, thermal nuclei "
                                        "kT=0.01 around the restraint centres",
                            "value_is": "FP64 trajectory-steps/s, inputs resident; mixed under results"},
                    cpu_baseline={"value": cpu, "unit": UNIT, "cores": 1, "kind": "oracle",
                                  "sample": f"{ns} trajectories x 5 steps"},
                    mixed={"value": res["mixed"]["traj_steps_per_s"],
                           "dtype": "mixed (f32 coefficients, generator, propagation, LU and ratio "
                                    "solves; f64 eigenpairs, forces, probabilities, rescale)"},
                    results=res)
    elif args.workload == "syev":
        # the batched dense symmetric eigensolver (eigenvalues and eigenvectors)
        # and the two-orbital dynamics that takes its eigenpairs from it
        from paper_2212_00518_gb300 import two
        res = {}
        for n in (64, 102, 256):
            B = 4096 if n <= 102 else 1024
            A = W.random_symmetric(B, n, seed=n)
            for dtype, name in ((torch.float64, "fp64"), (torch.float32, "fp32")):
                tA = torch.tensor(A, dtype=dtype, device="cuda")
                lam = torch.empty((B, n), dtype=dtype, device="cuda")
                V = torch.empty((B, n, n), dtype=dtype, device="cuda")
                prec = P.PREC_FP64 if dtype == torch.float64 else P.PREC_MIXED
                work = torch.empty(P.iesh.load().iesh_syev_work_bytes(B, n, prec, 1), dtype=torch.uint8,
                                   device="cuda")
                ms = _timed_steps(torch, stream, lambda: P.iesh.syev_batched(tA, lam, V, work=work),
                                  args.warmup, args.steps)
                sec = ms / args.steps / 1e3
                flops = B * (8.0 / 3.0 + 6.0) * n ** 3  # reduction + P + about 6 n^3 for the rotations
                res[f"n{n}_{name}"] = {"matrices": B, "matrices_per_s": B / sec, "ms": 1e3 * sec,
                                       "approx_tflops": flops / sec / 1e12}
        n, dt = args.n_traj, 2.0
        md0 = W.two_orbital_profiled(100, seed=5)
        x, p, occ, C = W.two_orbital_state(md0, n, 3, kT=0.01, weight=0.5)
        dyn = {}
        for prec, solver, name in ((P.PREC_FP64, "nested", "fp64"), (P.PREC_MIXED, "nested", "mixed"),
                                   (P.PREC_FP64, "dense", "fp64_dense"), (P.PREC_MIXED, "dense", "mixed_dense")):
            md = dict(md0, eigensolver="dense") if solver == "dense" else md0
            c = two.TwoOrbitalContext(md, n, precision=prec, stream=stream.cuda_stream)
            c.set_state(x, p, occ.astype(np.int16), C if prec == P.PREC_FP64 else C.astype(np.complex64))
            c.run(dt, max(3, args.warmup), 0)
            c.profile(True)
            ms = _timed_steps(torch, stream, lambda: c.run(dt, 1, 0), 0, args.steps)
            prof = c.profile_read()
            c.profile(False)
            tot = sum(v[0] for v in prof.values())
            dyn[name] = {"traj_steps_per_s": n * args.steps / (ms / 1e3),
                         "kernel_share": {k: v[0] / tot for k, v in prof.items() if tot > 0},
                         "status_nonzero": int(np.count_nonzero(c.get_state()["status"]))}
            c.close()
        # textbook work of the symmetric QR algorithm with eigenvectors, 9 n^3
        # flops per matrix (tridiagonalisation, forming P, the QL rotations)
        r102 = res["n102_fp64"]
        ach = r102["matrices"] * 9.0 * 102 ** 3 / (r102["ms"] / 1e3) / 1e12
        roof = {"bound": "alu", "kernel": "iesh_syev_batched n=102 FP64 (k_syev_reduce + k_syev_qlv + "
                                          "k_syev_out, one call timed with CUDA events)",
                "achieved": ach, "peak": FP64_NOMINAL_TFLOPS, "unit": "TFLOP/s",
                "frac": ach / FP64_NOMINAL_TFLOPS,
                "achieved_is": "9 n^3 flops per matrix (symmetric QR with eigenvectors) x matrices / "
                               "call time",
                "peak_source": "derived: 2 DFMA/clk/SM x 152 SMs x 2.07 GHz",
                "traffic": None,
                "traffic_source": "not per call: the ncu capture of k_syev_qlv alone is summarised "
                                  "with the eigensolver profile"}
        line.update(metric="batched dense symmetric eigensolver, matrices/s (eigenvalues + eigenvectors)",
                    unit="matrices/s", value=res["n102_fp64"]["matrices_per_s"], dtype="f64", roofline=roof,
                    config={"workload": "random symmetric matrices n in {64, 102, 256} (4096, 4096, 1024 "
                                        "per batch), FP64 and FP32; two-orbital dynamics with own bath "
                                        f"profiles (non-parallel couplings), 100 GL states, {n} trajectories, "
                                        "dt=2, eigenpairs from two nested secular equations (default) "
                                        "and from the dense solver",
                            "value_is": "n=102 FP64 matrices/s"},
                    results={"syev": res, "two_orbital_profiled": dyn})
    elif args.workload == "eocc":
        from paper_2212_00518_gb300 import eocc as E
        wl = W.eocc_workload(M=300, B=65536, seed=5)
        model = E.EOccModel(wl, stream=stream.cuda_stream)
        out = {}
        for dtype in (torch.float32, torch.float64):
            x = torch.tensor(wl["x"], device="cuda", dtype=dtype)
            th = torch.tensor(wl["theta"], device="cuda", dtype=dtype)
            gE = torch.ones(65536, device="cuda", dtype=dtype)

            def step():
                _, saved, _ = model.forward(x, th)
                model.backward(x, th, saved, gE)
            ms = _timed_steps(torch, stream, step, args.warmup, args.steps)
            out[str(dtype).split(".")[-1]] = 65536 * args.steps / (ms / 1e3)
        line.update(metric="E_occ forward + backward geometries/s", unit="geometries/s",
                    value=out["float32"], dtype="f32",
                    config={"workload": "two adsorbate orbitals, M=300 bath states, Ne=151, six "
                                        "coordinates, 16 parameters, 65536 geometries"},
                    results={"float32": out["float32"], "float64": out["float64"]})
    print(json.dumps(line), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--M", type=int, default=100)
    ap.add_argument("--n-traj", dest="n_traj", type=int, default=4096)
    ap.add_argument("--dt", type=float, default=1.0)
    ap.add_argument("--seed", type=int, default=0)
    ap.add_argument("--e2e-steps", dest="e2e_steps", type=int, default=3)
    ap.add_argument("--e2e-chunks", dest="e2e_chunks", type=int, default=4,
                    help="trajectory ranges of iesh_run_host in the end-to-end leg")
    ap.add_argument("--cpu-steps", dest="cpu_steps", type=int, default=400)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-mixed", action="store_true")
    ap.add_argument("--no-config3", dest="no_config3", action="store_true",
                    help="skip the M=200, Ne=100 comparison (FP64 and mixed)")
    ap.add_argument("--c3-traj", dest="c3_traj", type=int, default=8192)
    ap.add_argument("--skip-bound", dest="skip_bound", action="store_true",
                    help="skip the ratio solves when the exact hop-probability bound is below "
                         "the uniform (Sec. II C; hop decisions unchanged)")
    ap.add_argument("--no-overlap", action="store_true",
                    help="skip the diabatic-basis propagator variant")
    ap.add_argument("--workload", choices=["dw", "paper", "scatter", "erpenbeck", "relaxation", "eocc",
                                           "two", "syev"],
                    default="dw",
                    help="dw: the double-well batch (default, --M/--n-traj); the others print "
                         "secondary measurements")
    ap.add_argument("--autotune", action="store_true")
    ap.add_argument("--no-deflation", dest="no_deflation", action="store_true",
                    help="run the Chebyshev series over the whole spectrum interval (no deflation "
                         "of the isolated top level)")
    args = ap.parse_args()
    if args.impl == "reference":
        run_reference(args)
    elif args.workload != "dw":
        run_workload(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
