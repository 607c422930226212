#!/usr/bin/env python
"""RT-TDA benchmark: trajectory-steps/s of the batched sigma build + RK4 stepper.

Workload (linear absorption): nocc=64, nvirt=448, naux=1536 (dim 28673),
synthetic factors (seeded generator), three trajectories kicked along x, y, z
(kappa = 1e-3) from |0>, RK4 dt = 0.05 au.  One "step" is one RK4 step of the
whole batch (four sigma builds per trajectory, observables included).

Default: 1 GPU.  Under torchrun each rank propagates its own batch (weak
scaling, no data-path collective); timing is the max over ranks.
`--impl reference` times the CPU oracle on a bounded row sample instead.
"""
from __future__ import annotations

import argparse
import json
import os
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "RT-TDA trajectory-steps/s vs plain FP64 path at stated dipole err; p50/p99 latency"
UNIT = "trajectory-steps/s"
CX, KAPPA, SEED = 0.2, 1e-3, 0
DIRS = [(1.0, 0.0, 0.0), (0.0, 1.0, 0.0), (0.0, 0.0, 1.0)]
# workloads: the linear-absorption one is the default bench line; the others
# are the batched field scan and the large system
WORKLOADS = {
    "absorption": dict(nocc=64, nvirt=448, naux=1536, dt=0.05,
                       desc="linear absorption: 3 trajectories (x/y/z kicks, kappa=1e-3) per GPU"),
    "fieldscan": dict(nocc=128, nvirt=768, naux=3072, dt=0.04,
                      desc=("batched field scan: 32 sin^2 pulses (400 au) per GPU at omega = lambda_min(A) and "
                            "lambda_min/2, amplitudes log-spaced 1e-3..5e-2, z-polarised")),
    "large": dict(nocc=256, nvirt=1536, naux=4096, dt=0.05, desc="large system: one z kick kappa=1e-3"),
    # the shape of the paper's smallest timing system (Indigo: 68 occupied, 252
    # virtual orbitals) with a synthetic RI basis of 3 x 320 functions, driven
    # by the timing study's pulse; context only (the paper's sigma is an
    # AO-direct build, not this RI-factorised one)
    "paper_timing": dict(nocc=68, nvirt=252, naux=960, dt=0.05,
                         desc=("paper timing-study shape: one transform-limited pulse, 2.5 eV carrier, "
                               "5e11 W/cm2 peak, FWHM 0.91 fs, centred at 50 au")),
}
NOCC, NVIRT, NAUX, DT = 64, 448, 1536, 0.05
NDIM = 1 + NOCC * NVIRT
WORKLOAD = ""


def set_workload(name: str, naux: int = 0) -> None:
    global NOCC, NVIRT, NAUX, DT, NDIM, WORKLOAD
    w = WORKLOADS[name]
    NOCC, NVIRT, NAUX, DT = w["nocc"], w["nvirt"], naux or w["naux"], w["dt"]
    NDIM = 1 + NOCC * NVIRT
    WORKLOAD = (f"{w['desc']}: nocc={NOCC} nvirt={NVIRT} naux={NAUX} (dim {NDIM}), RK4 dt={DT} au, c_x={CX}")


set_workload("absorption")


def lowest_eigenvalue(rb, mol, iters=60):
    """lambda_min of A by Lanczos with full reorthogonalisation, using the
    library's sigma (a kicked trajectory has E = 0 for t > 0, so sigma = A c)."""
    import torch
    prop = rb.Propagator(mol, CX, "bf16x3")
    prop.set_field([dict(kind=rb.KICK, E0=KAPPA, direction=(0.0, 0.0, 1.0))])
    n = prop.n
    rng = np.random.default_rng(7)
    q = rng.standard_normal(n)
    q[0] = 0.0
    q /= np.linalg.norm(q)
    Q, alpha, beta = [q], [], []
    cd = torch.zeros((1, n, 2), dtype=torch.float64, device="cuda")
    sd = torch.zeros_like(cd)
    for k in range(iters):
        cd[0, :, 0] = torch.from_numpy(Q[-1])
        cd[0, :, 1] = 0.0
        rb.rttda_sigma(prop.h, cd.data_ptr(), 1.0, sd.data_ptr(), 0)
        rb.rttda_sync(prop.h)
        w = sd[0, :, 0].cpu().numpy()
        a = float(w @ Q[-1])
        w = w - a * Q[-1] - (beta[-1] * Q[-2] if beta else 0.0)
        for qq in Q:
            w -= (w @ qq) * qq
        alpha.append(a)
        b = float(np.linalg.norm(w))
        if b < 1e-12 or k == iters - 1:
            break
        beta.append(b)
        Q.append(w / b)
    prop.close()
    Tm = np.diag(alpha) + np.diag(beta[:len(alpha) - 1], 1) + np.diag(beta[:len(alpha) - 1], -1)
    return float(np.linalg.eigvalsh(Tm)[0])


def workload_pulses(rb, name, mol):
    if name == "fieldscan":
        lam = lowest_eigenvalue(rb, mol)
        amps = np.exp(np.linspace(np.log(1e-3), np.log(5e-2), 16))
        return [dict(kind=rb.SIN2, E0=float(a), omega=w, duration=400.0, direction=(0.0, 0.0, 1.0))
                for w in (lam, 0.5 * lam) for a in amps], {"lambda_min": lam}
    if name == "large":
        return [dict(kind=rb.KICK, E0=KAPPA, direction=(0.0, 0.0, 1.0))], {}
    if name == "paper_timing":
        ev = 1.0 / 27.211386245988                   # Hartree per eV
        fs = 1.0 / 2.4188843265857e-2                # au of time per fs
        E0 = float(np.sqrt(5e11 / 3.50944758e16))    # peak field from the intensity (au)
        return [dict(kind=rb.GAUSS_TL, E0=E0, omega=2.5 * ev, t0=50.0, fwhm=0.91 * fs,
                     direction=(0.0, 0.0, 1.0))], {"E0_au": E0}
    return [dict(kind=rb.KICK, E0=KAPPA, direction=d) for d in DIRS], {}
PEAKS_FILE = os.path.join(ROOT, "MEASURED_PEAKS.json")


def dist_info():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


class Ranks:
    """Process-group plumbing of a multi-GPU run.  Every rank propagates its
    own batch (weak scaling); the only cross-rank operations are a barrier
    around the timed region and the maximum of the timed seconds."""

    def __init__(self, backend: str = "nccl", device: str = "cuda"):
        import torch
        self.torch = torch
        self.rank, self.world, self.local = dist_info()
        self.device = device
        if self.world > 1:
            import torch.distributed as dist
            kw = {"device_id": torch.device("cuda", self.local)} if backend == "nccl" else {}
            dist.init_process_group(backend, **kw)

    def barrier(self) -> None:
        if self.world > 1:
            self.torch.distributed.barrier()

    def max(self, x: float) -> float:
        if self.world == 1:
            return x
        t = self.torch.tensor([x], dtype=self.torch.float64, device=self.device)
        self.torch.distributed.all_reduce(t, op=self.torch.distributed.ReduceOp.MAX)
        return float(t.item())

    def aggregate_rate(self, units_per_rank: float, seconds: float) -> float:
        """Whole-job throughput: all ranks' units over the slowest rank's time."""
        return self.world * units_per_rank / self.max(seconds)

    def close(self) -> None:
        if self.world > 1:
            self.torch.distributed.destroy_process_group()


def base_config(prec: str, world: int, T: int = 3) -> dict:
    return {"workload": WORKLOAD, "precision": prec, "trajectories_per_gpu": T,
            "global_trajectories": T * world, "parallelism": f"trajectory replicas x{world}",
            "l2": "inputs larger than L2: every stage streams the B_vv planes (>1 GB) and B_ov",
            "seed": SEED}


# ---------------------------------------------------------------------------
# CPU oracle sample (cpu_baseline and --impl reference)
# ---------------------------------------------------------------------------
class OracleSample:
    """Dense sigma = H(t)c of the oracle on a block of rows of the explicit A.

    The block is the rows of the first `nocc_rows` occupied orbitals (all
    virtuals); one sampled step is the oracle's sigma on that block for all
    three trajectories, four times (one RK4 step), and the full step is that
    time scaled by (rows of A) / (rows in the block).  Building A is setup,
    as rttda_create is for the GPU."""

    def __init__(self, mol, nocc_rows: int):
        from oracle import rttda_oracle as orc
        self.orc = orc
        self.rows = np.arange(1, 1 + nocc_rows * NVIRT)
        self.A = orc.A_block(mol, CX, 0, nocc_rows)
        self.M = [orc.M_rows(*orc.dipole_along(mol, d), self.rows) for d in DIRS]
        rng = np.random.default_rng(1)
        self.c = [rng.standard_normal(NDIM) + 1j * rng.standard_normal(NDIM) for _ in DIRS]

    def step(self):
        for k in range(3):
            c = self.c[k]
            for _ in range(4):
                sg = self.orc.sigma(self.A, self.M[k], 0.0, c)
                c[self.rows] = c[self.rows] + (-1j * DT) * sg * 1e-6

    def scale(self) -> float:
        return NDIM / len(self.rows)

    @staticmethod
    def cores() -> int:
        try:
            from threadpoolctl import threadpool_info
            n = [i.get("num_threads", 1) for i in threadpool_info() if i.get("user_api") == "blas"]
            return max(n) if n else 1
        except Exception:
            return 1


def time_oracle(mol, nocc_rows: int, nsteps: int, warmup: int = 1):
    s = OracleSample(mol, nocc_rows)
    for _ in range(warmup):
        s.step()
    t0 = time.perf_counter()
    for _ in range(nsteps):
        s.step()
    dt_sample = (time.perf_counter() - t0) / nsteps
    full_step = dt_sample * s.scale()
    return {"value": 3.0 / full_step, "unit": UNIT, "cores": OracleSample.cores(), "kind": "oracle",
            "sample": (f"oracle dense sigma on {len(s.rows)} of {NDIM} rows of A (occupied 0..{nocc_rows - 1}), "
                       f"3 trajectories x 4 sigma per step, {nsteps} sampled steps, scaled x{s.scale():.2f} "
                       "to a full RK4 step; building A excluded as setup"),
            "ms_per_step": full_step * 1e3}


def run_reference(args):
    rank, world, _ = dist_info()
    if rank != 0:
        return 0
    from paper_2601_16949_b300 import synth
    mol = synth.molecule(NOCC, NVIRT, NAUX, seed=SEED)
    base = time_oracle(mol, 2, args.steps, warmup=args.warmup)
    line = {"metric": METRIC, "value": base["value"], "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": base["ms_per_step"], "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": base_config("fp64 (CPU oracle)", 1), "impl": "reference",
            "cpu_baseline": {k: base[k] for k in ("value", "unit", "cores", "kind", "sample")},
            "e2e": {"value": base["value"], "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


# ---------------------------------------------------------------------------
# Clock sampling during the timed region
# ---------------------------------------------------------------------------
class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, uuid: str | None):
        self.uuid = uuid
        self.proc = None

    def __enter__(self):
        cmd = ["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits", "-lms", "200"]
        if self.uuid:
            cmd += ["-i", self.uuid]
        try:
            self.proc = subprocess.Popen(cmd, stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except Exception:
            self.proc = None
        return self

    def __exit__(self, *exc):
        self.out = ""
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.out, _ = self.proc.communicate(timeout=5)
            except Exception:
                self.proc.kill()
                self.out = ""

    def summary(self) -> dict:
        sm, mx, reasons = [], [], set()
        names = ("hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap")
        for line in (self.out or "").splitlines():
            f = [x.strip() for x in line.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                mx.append(float(f[2]))
            except ValueError:
                continue
            for nm, val in zip(names, f[5:9]):
                if val.lower().startswith("active"):
                    reasons.add(nm)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": [], "samples": 0}
        return {"sm_mhz": float(np.median(sm)), "sm_max_mhz": max(mx), "reasons": sorted(reasons),
                "samples": len(sm)}


# ---------------------------------------------------------------------------
# Roofline: algorithmic work per launch of a kernel class
# ---------------------------------------------------------------------------
PREC_INFO = {  # factor bytes, exchange planes, tensor products per K tile
    "fp64": dict(fb=8, planes=1, nprod=1, tensor=False),
    "fp32": dict(fb=4, planes=1, nprod=1, tensor=False),
    "bf16": dict(fb=2, planes=1, nprod=1, tensor=True),
    "bf16x3": dict(fb=4, planes=2, nprod=3, tensor=True),
    "bf16x2": dict(fb=4, planes=2, nprod=2, tensor=True, zplanes=1),
    # Ozaki digits: 6 BF16 digit planes per operand, 21 digit pairs per K tile
    "fp64oz": dict(fb=8, planes=6, nprod=21, tensor=True, zplanes=6),
}


# DRAM bytes (dram__bytes_read.sum + dram__bytes_write.sum) of one launch of
# the dominant kernel, from one ncu --set full capture of that kernel on this
# workload.  Keyed by (workload, precision, kernel class, main kernel kind
# (2 wide-M, 4 transposed), BN, MB, K tile):
# the number holds only for that kernel and plan.
PROFILED_TRAFFIC = {
    ("absorption", "bf16x2", "exchange_main", 4, 192, 2, 32): 1.766175e9 + 3.553792e6,
}


def algorithmic_work(prec: str, cls: str, T: int):
    """(flop, bytes) of one launch of a kernel class on this workload.

    exchange_main: sum_{P,b} Z^P_(col,i),b B^P_ab, M = 2T*nocc, N = nvirt,
    K = naux*nvirt; bytes = Z and B_vv read once (all planes).  Flops count
    every tensor product of the split (nprod x 2MNK)."""
    pi = PREC_INFO[prec]
    C = 2 * T
    o, v, P = NOCC, NVIRT, NAUX
    if cls == "exchange_main":
        M, N, K = C * o, v, P * v
        eb = 2 if pi["tensor"] else pi["fb"]
        zp = pi.get("zplanes", pi["planes"])
        return pi["nprod"] * 2.0 * M * N * K, eb * (zp * M * K + pi["planes"] * P * v * v)
    if cls == "coulomb":
        return 2 * 2.0 * P * o * v * C, 2.0 * P * o * v * (pi["fb"] if prec != "bf16x3" else 4)
    if cls == "exchange_z" and prec == "fp64oz":
        # Z build into int64 Z (written, read back by the digit split) plus
        # its 6 BF16 digits; digits of B_oo and of the amplitudes read once
        nz = P * o * v * C
        return pi["nprod"] * 2.0 * P * o * o * v * C, (8 + 8 + 2 * 6) * nz + 2 * 6 * (P * o * o + o * v * C)
    if cls == "exchange_z":
        eb = 2 if pi["tensor"] else pi["fb"]
        zp = pi.get("zplanes", pi["planes"])
        nz = 3 if prec in ("bf16x3", "bf16x2") else pi["nprod"]
        return nz * 2.0 * P * o * o * v * C, eb * (zp * P * o * v * C + pi["planes"] * P * o * o)
    return None, None


def roofline(prec: str, cls: str, prof_entry, T: int, peaks: dict, nsigma: int) -> dict:
    """Roofline of one kernel class.  The unit is one sigma build (one RK4
    stage): when the exchange is chunked over P, a stage is several launches
    of the class, so work and time are both taken per stage (the sum over
    its launches), which keeps achieved = work / duration for any chunking.

    The class is timed inside a long run of steps, so the tensor peak is the
    sustained (power-capped) measured bf16 rate; the burst rate is reported
    beside it."""
    ms, n = prof_entry
    flop, byts = algorithmic_work(prec, cls, T)
    hbm = peaks.get("hbm_gbs", 6400.0)
    bf16_burst = peaks.get("bf16_tflops", 1800.0)
    bf16 = peaks.get("bf16_tflops_sustained", 1400.0)
    out = {"kernel": cls, "unit_of_work": "one sigma build (all launches of the class in one RK4 stage)",
           "avg_launch_ms": ms / max(n, 1), "launches_timed": n, "sigma_builds_timed": nsigma,
           "launches_per_sigma": n / max(nsigma, 1), "ms_per_sigma": ms / max(nsigma, 1), "traffic": None,
           "flop_per_sigma": flop, "bytes_per_sigma": byts}
    if flop is None or n == 0:
        out.update({"bound": None, "achieved": None, "peak": None, "unit": None, "frac": None})
        return out
    sec = ms / nsigma / 1e3
    pi = PREC_INFO[prec]
    if pi["tensor"]:
        cpeak, cunit = bf16, "TFLOP/s"
        csrc = "of measured: bf16 sustained (MEASURED_PEAKS.json bf16_tflops_sustained)"
        cbound = "tensor"
    else:
        lanes = 128 if prec == "fp32" else 64
        cpeak = 148 * lanes * 2 * 2.032e9 / 1e12
        cunit, cbound = "TFLOP/s", "alu"
        csrc = f"derived: 148 SM x {lanes} {'FP32' if prec == 'fp32' else 'FP64'} FMA/clk x 2 x 2032 MHz"
    t_comp = flop / (cpeak * 1e12)
    t_mem = byts / (hbm * 1e9)
    if t_mem >= t_comp:
        out.update({"bound": "hbm", "achieved": byts / sec / 1e9, "peak": hbm, "unit": "GB/s",
                    "peak_source": "of measured: HBM copy (MEASURED_PEAKS.json hbm_gbs)"})
    else:
        out.update({"bound": cbound, "achieved": flop / sec / 1e12, "peak": cpeak, "unit": cunit,
                    "peak_source": csrc})
    out["frac"] = out["achieved"] / out["peak"]
    out["other_bound_frac"] = (flop / sec / 1e12 / cpeak) if out["bound"] == "hbm" else (byts / sec / 1e9 / hbm)
    if pi["tensor"]:
        out["tensor_frac_of_burst"] = flop / sec / 1e12 / bf16_burst
    return out


# ---------------------------------------------------------------------------
# GPU arm
# ---------------------------------------------------------------------------
def run_gpu(args):
    import torch
    rank, world, local = dist_info()
    torch.cuda.set_device(local)
    ranks = Ranks("nccl", "cuda")
    from paper_2601_16949_b300 import binding as rb
    from paper_2601_16949_b300 import synth
    barrier, max_over_ranks = ranks.barrier, ranks.max

    if args.workload in ("large", "fieldscan"):
        # FP64 factors of this size take minutes to draw on the host (or do
        # not fit there): draw them on the GPU
        mol = synth.molecule_device(NOCC, NVIRT, NAUX, seed=SEED)
        args.no_cpu_baseline = True
    else:
        mol = synth.molecule(NOCC, NVIRT, NAUX, seed=SEED)
    pulses, wl_info = workload_pulses(rb, args.workload, mol)
    T, K, W = len(pulses), args.steps, args.warmup
    prop = rb.Propagator(mol, CX, args.prec, integrator=args.integrator)
    prop.set_field(pulses)
    h = prop.h
    pop_info = None
    if args.populations > 0:
        # TI-TDA states by Davidson on the library's sigma (set-up, timed
        # apart), then their overlaps recorded at every timed step
        t0 = time.perf_counter()
        w_st, X_st, it_st = prop.eigenstates(args.populations, tol=1e-5, max_iter=300)
        pop_info = {"states": args.populations, "eigensolver_s": time.perf_counter() - t0,
                    "davidson_iterations": it_st, "lowest_excitation_ha": float(w_st[0]),
                    "recorded": "overlaps with every state at every step, inside the timed region"}
        prop.set_projectors(X_st)
        if args.autocorrelation:
            pop_info["autocorrelation"] = "recorded at every step, inside the timed region"
    if args.autocorrelation:
        rb.rttda_set_autocorrelation(h, True)
    dev = torch.device("cuda", local)
    c_out = torch.zeros((T, NDIM, 2), dtype=torch.float64, device=dev)
    dip = torch.zeros((T, K + 1), dtype=torch.float64, device=dev)
    nrm = torch.zeros((T, K + 1), dtype=torch.float64, device=dev)
    # a dedicated stream: the library's kernels and the timing events must
    # share it (the legacy default stream would not order with the library)
    stream = torch.cuda.Stream(device=dev)
    torch.cuda.set_stream(stream)
    sptr = stream.cuda_stream

    def propagate(nsteps, d, n):
        rb.rttda_propagate_device(h, 0, DT, nsteps, c_out.data_ptr(), d.data_ptr(), n.data_ptr(), sptr)

    # warm-up (>= 3 steps)
    wd = torch.zeros((T, W + 1), dtype=torch.float64, device=dev)
    wn = torch.zeros_like(wd)
    propagate(W, wd, wn)
    torch.cuda.synchronize()

    uuid = None
    try:
        uuid = "GPU-" + str(torch.cuda.get_device_properties(local).uuid)
    except Exception:
        pass
    plan = rb.rttda_plan(h)
    launches0, _ = rb.rttda_launch_stats(h)
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    with ClockSampler(uuid) as clk:
        barrier()
        torch.cuda.synchronize()
        ev0.record(stream)
        propagate(K, dip, nrm)
        ev1.record(stream)
        torch.cuda.synchronize()
        barrier()
    launches1, per_step = rb.rttda_launch_stats(h)
    rb.rttda_sync(h, sptr)
    ms = max_over_ranks(ev0.elapsed_time(ev1))
    value = world * T * K / (ms / 1e3)
    dip32 = dip.cpu().numpy()
    if args.only_timed:
        if rank == 0:
            print(json.dumps({"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": K,
                              "warmup": W, "ms_per_step": ms / K, "mode": "only-timed", "prec": args.prec}))
        prop.close()
        ranks.close()
        return 0

    # per-kernel timing pass (events around every kernel class, same workload)
    rb.rttda_profile(h, True)
    kp = min(K, 40)
    pd_, pn_ = torch.zeros((T, kp + 1), dtype=torch.float64, device=dev), torch.zeros((T, kp + 1), dtype=torch.float64, device=dev)
    propagate(kp, pd_, pn_)
    torch.cuda.synchronize()
    prof = rb.rttda_profile_read(h)
    rb.rttda_profile(h, False)

    # plain FP64 single-trajectory path on the same molecule (the batch's
    # last trajectory)
    p64 = rb.Propagator(mol, CX, "fp64", integrator=args.integrator)
    p64.set_field([pulses[-1]])
    k64 = max(2, min(args.fp64_steps, K))
    d64 = torch.zeros((1, k64 + 1), dtype=torch.float64, device=dev)
    n64 = torch.zeros_like(d64)
    c64 = torch.zeros((1, NDIM, 2), dtype=torch.float64, device=dev)
    rb.rttda_propagate_device(p64.h, 0, DT, 1, c64.data_ptr(), d64.data_ptr(), n64.data_ptr(), sptr)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    rb.rttda_propagate_device(p64.h, 0, DT, k64, c64.data_ptr(), d64.data_ptr(), n64.data_ptr(), sptr)
    e1.record(stream)
    torch.cuda.synchronize()
    fp64_rate = k64 / (e0.elapsed_time(e1) / 1e3)
    d64h = d64.cpu().numpy()[0]
    ref = d64h - d64h[0]
    dip_err = float(np.max(np.abs(dip32[T - 1, :k64 + 1] - d64h)) / max(np.max(np.abs(ref)), 1e-300))
    p64.close()

    # end to end through the host-buffer ABI: per step, H2D of the state from
    # pinned memory (rttda_set_state), one RK4 step, D2H of state and traces
    ke = max(3, min(args.e2e_steps, K))
    pin = lambda *s: torch.zeros(s, dtype=torch.float64).pin_memory()
    ch, co, dh, nh = pin(T, NDIM, 2), pin(T, NDIM, 2), pin(T, 2), pin(T, 2)
    tcur = rb.rttda_get_state(h, ch.numpy())
    rb.rttda_set_state(h, ch.data_ptr(), tcur)
    rb.rttda_resume(h, DT, 1, co.data_ptr(), dh.data_ptr(), nh.data_ptr())
    barrier()
    t0 = time.perf_counter()
    for _ in range(ke):
        rb.rttda_set_state(h, ch.data_ptr(), tcur)
        rb.rttda_resume(h, DT, 1, co.data_ptr(), dh.data_ptr(), nh.data_ptr())
        ch, co = co, ch
        tcur += DT
    e2e_s = max_over_ranks(time.perf_counter() - t0)
    e2e = {"value": world * T * ke / e2e_s, "unit": UNIT,
           "h2d_bytes_per_step": T * NDIM * 16, "d2h_bytes_per_step": T * NDIM * 16 + 2 * T * 2 * 8,
           "steps": ke, "call": "rttda_set_state + rttda_resume(nsteps=1) per step, pinned host buffers"}

    # roofline of the dominant kernel class
    peaks = json.load(open(PEAKS_FILE)) if os.path.exists(PEAKS_FILE) else {}
    ms_cls = {k: v[0] for k, v in prof.items()}
    dom = max(ms_cls, key=ms_cls.get)
    # sigma builds in the profiled call: 4 per RK4 step; 2 per split-operator
    # step plus the call's first half step
    nsig = 4 * kp if args.integrator == "rk4" else 2 * kp + 1
    roof = roofline(args.prec, dom, prof[dom], T, peaks, nsig)
    tkey = (args.workload, args.prec, dom, plan["main_kernel"], plan["main_bn"], plan["main_mb"], plan["main_kb"])
    if tkey in PROFILED_TRAFFIC and plan["z_chunk"] >= NAUX:
        roof["traffic"] = PROFILED_TRAFFIC[tkey]
        roof["traffic_source"] = "ncu capture of this kernel and plan (one launch = one sigma build)"
    roof["class_ms_share"] = {k: round(v / max(sum(ms_cls.values()), 1e-30), 4) for k, v in ms_cls.items()}
    roof["class_ms_per_step"] = {k: round(v / kp, 4) for k, v in ms_cls.items()}

    cpu = None
    if rank == 0 and not args.no_cpu_baseline:
        # row block of the explicit A of at most ~1 GB
        rows_occ = int(max(1, min(8, (1 << 27) // (NVIRT * NDIM))))
        cb = time_oracle(mol, rows_occ, args.cpu_steps, warmup=1)
        cpu = {k: cb[k] for k in ("value", "unit", "cores", "kind", "sample")}

    dtype = {"fp64": "f64", "fp32": "f32", "bf16": "bf16", "bf16x3": "bf16x3", "bf16x2": "bf16x2",
             "fp64oz": "f64 (exchange: Ozaki BF16 digits)"}[args.prec]
    cfg = base_config(args.prec, world, T)
    if pop_info:
        cfg["populations"] = pop_info
    elif args.autocorrelation:
        cfg["autocorrelation"] = "recorded at every step, inside the timed region"
    cfg["integrator"] = {"rk4": "classical RK4 (4 sigma builds per step)",
                         "sso": "symplectic split operator (2 sigma builds per step)"}[args.integrator]
    cfg.update(wl_info)
    cfg.update({"fp64_path_traj_steps_per_s": fp64_rate, "speedup_vs_fp64_path": value / world / fp64_rate,
                "fp64_path": f"plain FP64, one trajectory (the batch's last), {k64} timed steps",
                "dipole_rel_err_vs_fp64": dip_err, "dipole_err_horizon_steps": k64,
                "launches_per_step": per_step, "plan": plan})
    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": K, "warmup": W,
            "ms_per_step": ms / K, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": dtype, "data": "synthetic", "config": cfg, "roofline": roof, "cpu_baseline": cpu,
            "e2e": e2e, "gpu_launches": int(launches1 - launches0), "clocks": clk.summary()}
    if rank == 0:
        print(json.dumps(line), flush=True)
    prop.close()
    ranks.close()
    return 0


def run_accuracy(args):
    """Long-horizon dipole / norm error of each precision against FP64 on the
    same molecule, one z-kicked trajectory."""
    import torch
    from paper_2601_16949_b300 import binding as rb
    from paper_2601_16949_b300 import synth
    torch.cuda.set_device(0)
    mol = synth.molecule(NOCC, NVIRT, NAUX, seed=SEED)
    pulse = [dict(kind=rb.KICK, E0=KAPPA, direction=(0.0, 0.0, 1.0))]
    n = args.accuracy
    ref_prec = args.accuracy_ref
    res = {}
    for prec in [ref_prec] + [p for p in args.accuracy_precs.split(",") if p and p != ref_prec]:
        pr = rb.Propagator(mol, CX, prec)
        pr.set_field(pulse)
        t0 = time.perf_counter()
        _, dip, nrm = pr.propagate(DT, n, want_state=False)
        res[prec] = (dip[0], nrm[0], time.perf_counter() - t0)
        pr.close()
    d64, n64, _ = res[ref_prec]
    ref = d64 - d64[0]
    out = {"mode": "accuracy", "reference": ref_prec, "workload": WORKLOAD, "steps": n, "horizon_au": n * DT,
           "trajectory": "z kick", "reference_norm_drift": float(np.max(np.abs(n64 - n64[0]))), "results": {}}
    for prec, (d, nr, sec) in res.items():
        if prec == ref_prec:
            continue
        err = np.abs(d - d64) / np.max(np.abs(ref))
        k = np.arange(len(err))
        out["results"][prec] = {
            "dipole_rel_err": float(np.max(err)),
            "dipole_rel_err_at": {str(int(m)): float(np.max(err[: m + 1]))
                                  for m in (n // 16, n // 8, n // 4, n // 2, n)},
            "norm_diff_vs_reference": float(np.max(np.abs(nr - n64))),
            "seconds": sec}
        del k
    out["reference_seconds"] = res[ref_prec][2]
    print(json.dumps(out), flush=True)
    return 0


def run_serving(args):
    """Continuous-batching trace (scaled-down serving workload): Poisson
    arrivals, a random molecule, pulse and length per request, admitted by
    footprint; reports p50/p99 time-to-spectrum and trajectory-steps/s."""
    import torch
    from paper_2601_16949_b300 import binding as rb
    from paper_2601_16949_b300 import synth
    torch.cuda.set_device(0)
    rng = np.random.default_rng(args.serving_seed)
    n = args.serving_requests
    arrivals = np.cumsum(rng.exponential(1.0 / args.serving_rate, n))
    spec = dict(gamma=1e-3, wmin=0.1, wmax=3.0, nfreq=512)
    reqs = []
    for k in range(n):
        while True:
            o = int(rng.integers(16, 49))
            v = int(rng.integers(64, 193))
            if v >= 4 * o:
                break
        P = 4 * v
        steps = int(rng.integers(200, 2001))
        if rng.random() < 0.5:
            pulse = dict(kind=rb.KICK, E0=1e-3, direction=(0.0, 0.0, 1.0))
        else:
            pulse = dict(kind=rb.SIN2, E0=float(np.exp(rng.uniform(np.log(1e-3), np.log(5e-2)))),
                         omega=float(rng.uniform(0.4, 2.5)), duration=0.8 * steps * DT, direction=(0.0, 0.0, 1.0))
        mol = synth.molecule(o, v, P, seed=1000 + k)
        reqs.append((mol, rb.make_request(mol, CX, args.prec, pulse, DT, steps, **spec), steps))
    srv = rb.rttda_server_create(int(args.serving_budget_gb * (1 << 30)), args.serving_slots, args.serving_chunk)
    ids = []
    t0 = time.perf_counter()
    for k, (mol, q, steps) in enumerate(reqs):
        delay = arrivals[k] - (time.perf_counter() - t0)
        if delay > 0:
            time.sleep(delay)
        ids.append(rb.rttda_server_submit(srv, q))
    for rid in ids:
        rb.rttda_server_wait(srv, rid, 3600.0)
    wall = time.perf_counter() - t0
    st = rb.rttda_server_stats_get(srv)
    states = [rb.rttda_server_poll(srv, rid)[0] for rid in ids]
    rb.rttda_server_destroy(srv)
    line = {"mode": "serving", "metric": "time-to-spectrum p50/p99 and trajectory-steps/s (continuous batching)",
            "requests": n, "arrival_rate_per_s": args.serving_rate, "precision": args.prec,
            "workload": ("scaled serving trace: nocc U[16,48], nvirt U[64,192] with nvirt >= 4 nocc, naux = 4 nvirt, "
                         "kick or sin^2 pulse (E0 log-uniform 1e-3..5e-2), 200-2000 RK4 steps, dt 0.05"),
            "completed": st["completed"], "failed": st["failed"], "all_done": all(x == rb.REQ_DONE for x in states),
            "p50_time_to_spectrum_s": st["p50_latency_s"], "p99_time_to_spectrum_s": st["p99_latency_s"],
            "mean_time_to_spectrum_s": st["mean_latency_s"],
            "trajectory_steps_per_s": st["trajectory_steps"] / max(st["busy_seconds"], 1e-9),
            "trajectory_steps": st["trajectory_steps"], "busy_seconds": st["busy_seconds"], "wall_seconds": wall,
            "max_concurrent": st["max_concurrent"], "slots": args.serving_slots,
            "budget_gb": args.serving_budget_gb, "chunk_steps": args.serving_chunk}
    print(json.dumps(line), flush=True)
    return 0


def main():
    ap = argparse.ArgumentParser(description=__doc__)
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=200)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="absorption", choices=sorted(WORKLOADS))
    ap.add_argument("--prec", default="bf16x2", choices=["fp64", "fp32", "bf16", "bf16x3", "bf16x2", "fp64oz"])
    ap.add_argument("--populations", type=int, default=0,
                    help="record overlaps with this many TI-TDA states (Davidson) at every step")
    ap.add_argument("--autocorrelation", action="store_true", help="record R(t) at every step")
    ap.add_argument("--integrator", default="rk4", choices=["rk4", "sso"],
                    help="time integrator of the timed propagation (the plain FP64 comparison path uses the same)")
    ap.add_argument("--accuracy", type=int, default=0,
                    help="instead of timing: propagate N steps with FP64 and the chosen precisions "
                         "(z kick) and print their dipole/norm errors against FP64")
    ap.add_argument("--accuracy-precs", default="fp32,bf16x3,bf16x2,bf16")
    ap.add_argument("--accuracy-ref", default="fp64")
    ap.add_argument("--serving", action="store_true", help="run the continuous-batching serving trace instead")
    ap.add_argument("--serving-requests", type=int, default=60)
    ap.add_argument("--serving-rate", type=float, default=5.0)
    ap.add_argument("--serving-slots", type=int, default=16)
    ap.add_argument("--serving-budget-gb", type=float, default=64.0)
    ap.add_argument("--serving-chunk", type=int, default=200)
    ap.add_argument("--serving-seed", type=int, default=5)
    ap.add_argument("--fp64-steps", type=int, default=4)
    ap.add_argument("--e2e-steps", type=int, default=30)
    ap.add_argument("--cpu-steps", type=int, default=3)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--naux", type=int, default=0,
                    help="override the workload's naux (smaller cases for profiler captures; not a bench line)")
    ap.add_argument("--only-timed", action="store_true",
                    help="warm-up and timed steps only (for profiler captures): no per-kernel pass, "
                         "no FP64 comparison, no end-to-end or CPU legs")
    args = ap.parse_args()
    args.warmup = max(3, args.warmup)   # at least three untimed warm-up steps
    set_workload(args.workload, args.naux)
    if args.gpus > 1 and "WORLD_SIZE" not in os.environ and args.impl == "ours":
        # one process per GPU: relaunch under torch.distributed.run
        import socket
        with socket.socket() as sk:
            sk.bind(("127.0.0.1", 0))
            port = sk.getsockname()[1]
        cmd = [sys.executable, "-m", "torch.distributed.run", "--nnodes=1", f"--nproc-per-node={args.gpus}",
               "--master-addr", "127.0.0.1", "--master-port", str(port), os.path.abspath(__file__)] + sys.argv[1:]
        return subprocess.call(cmd)
    if args.impl == "reference":
        return run_reference(args)
    if args.accuracy:
        return run_accuracy(args)
    if args.serving:
        return run_serving(args)
    return run_gpu(args)


if __name__ == "__main__":
    sys.exit(main())
