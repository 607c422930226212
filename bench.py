#!/usr/bin/env python
"""RT-TDA benchmark: trajectory-steps/s of the batched sigma build + RK4 stepper.

Default workload (the batched field scan): nocc=128, nvirt=768, naux=3072
(dim 98305), synthetic factors drawn on the GPU with a seeded generator,
32 trajectories driven by sin^2 pulses (400 au, z-polarised) at
omega = lambda_min(A) and lambda_min/2 with amplitudes log-spaced 1e-3 to
5e-2 au, RK4 dt = 0.04 au, plain BF16 factors with FP32 accumulation and an
FP64 amplitude state.  One "step" is one RK4 step of the whole batch (four
sigma builds per trajectory, observables included).  lambda_min(A) is the
lowest eigenvalue of the FP64-accurate sigma build (Davidson).

Other workloads (--workload): linear absorption (nocc=64, nvirt=448,
naux=1536, x/y/z kicks), the large system (nocc=256, nvirt=1536,
naux=4096, one z kick) and the shape of the paper's smallest timing system.

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
WORKLOADS = {
    "fieldscan": dict(nocc=128, nvirt=768, naux=3072, dt=0.04,
                      desc=("batched field scan: 32 sin^2 pulses (400 au) per GPU at omega = lambda_min(A) and "
                            "lambda_min/2, amplitudes log-spaced 1e-3..5e-2 au, z-polarised")),
    "absorption": dict(nocc=64, nvirt=448, naux=1536, dt=0.05,
                       desc="linear absorption: 3 trajectories (x/y/z kicks, kappa=1e-3) per GPU"),
    "large": dict(nocc=256, nvirt=1536, naux=4096, dt=0.05, desc="large system: one z kick kappa=1e-3"),
    # the shape of the paper's smallest timing system (Indigo: 68 occupied, 252
    # virtual orbitals) with a synthetic RI basis of 3 x 320 functions, driven
    # by the timing study's pulse; context only (the paper's sigma is an
    # AO-direct build, not this RI-factorised one)
    "paper_timing": dict(nocc=68, nvirt=252, naux=960, dt=0.05,
                         desc=("paper timing-study shape: one transform-limited pulse, 2.5 eV carrier, "
                               "5e11 W/cm2 peak, FWHM 0.91 fs, centred at 50 au")),
}
# workloads whose FP64 factors are drawn on the GPU (host generation takes
# minutes, or the factors do not fit in host memory)
DEVICE_FACTORS = ("fieldscan", "large")
NOCC = NVIRT = NAUX = NDIM = 0
DT = 0.0
WORKLOAD = NAME = ""


def set_workload(name: str, naux: int = 0) -> None:
    global NOCC, NVIRT, NAUX, DT, NDIM, WORKLOAD, NAME
    w = WORKLOADS[name]
    NOCC, NVIRT, NAUX, DT = w["nocc"], w["nvirt"], naux or w["naux"], w["dt"]
    NDIM = 1 + NOCC * NVIRT
    NAME = name
    WORKLOAD = (f"{w['desc']}: nocc={NOCC} nvirt={NVIRT} naux={NAUX} (dim {NDIM}), RK4 dt={DT} au, c_x={CX}")


set_workload("fieldscan")


def make_molecule(name: str, device: bool):
    from paper_2601_16949_b300 import synth
    if device:
        return synth.molecule_device(NOCC, NVIRT, NAUX, seed=SEED)
    return synth.molecule(NOCC, NVIRT, NAUX, seed=SEED)


def workload_pulses(name: str, lam: float | None = None):
    """The workload's pulses (binding pulse dicts; kinds as in rttda.h).
    The field scan needs lambda_min(A) (lam)."""
    if name == "fieldscan":
        amps = np.exp(np.linspace(np.log(1e-3), np.log(5e-2), 16))
        return [dict(kind=4, E0=float(a), omega=w, duration=400.0, direction=(0.0, 0.0, 1.0))
                for w in (lam, 0.5 * lam) for a in amps]
    if name == "large":
        return [dict(kind=0, E0=KAPPA, direction=(0.0, 0.0, 1.0))]
    if name == "paper_timing":
        ev = 1.0 / 27.211386245988                   # Hartree per eV
        fs = 1.0 / 2.4188843265857e-2                # au of time per fs
        E0 = float(np.sqrt(5e11 / 3.50944758e16))    # peak field from the intensity (au)
        return [dict(kind=2, E0=E0, omega=2.5 * ev, t0=50.0, fwhm=0.91 * fs, direction=(0.0, 0.0, 1.0))]
    return [dict(kind=0, E0=KAPPA, direction=d) for d in DIRS]


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


def base_config(prec: str, world: int, T: int) -> dict:
    return {"workload": WORKLOAD, "workload_name": NAME, "precision": prec, "trajectories_per_gpu": T,
            "global_trajectories": T * world, "parallelism": f"trajectory replicas x{world}",
            "l2": "inputs larger than L2: every stage streams the B_vv factors (>1 GB) and B_ov",
            "seed": SEED}


# ---------------------------------------------------------------------------
# CPU oracle sample (cpu_baseline and --impl reference)
# ---------------------------------------------------------------------------
def host_rows_molecule(mol, rows):
    """numpy copy of what the oracle needs for A_rows / M_rows on `rows`.
    Host molecules pass through.  From a GPU molecule: every array in full
    except B_vv, which is copied only at the virtual indices a of the sampled
    rows (A_rows reads B_vv[:, a, :] for those a alone); the rest of that
    array is never touched, so its zero pages are never allocated."""
    if not hasattr(mol["B_vv"], "is_cuda"):
        return mol
    out = {k: mol[k] for k in ("nocc", "nvirt", "naux")}
    for k in ("eps_occ", "eps_virt", "B_ov", "B_oo", "mu_oo", "mu_vv", "mu_0ov"):
        out[k] = mol[k].cpu().numpy()
    P, v = mol["naux"], mol["nvirt"]
    bvv = np.zeros((P, v, v))
    for a in sorted({(int(k) - 1) % v for k in rows if k > 0}):
        bvv[:, a, :] = mol["B_vv"][:, a, :].cpu().numpy()
    out["B_vv"] = bvv
    return out


class OracleSample:
    """The oracle's sigma = H(t)c on a sample of rows of the explicit A.

    `nrows` rows of the dim x dim matrices A and M_d (drawn uniformly with a
    fixed seed) are built from the definitions (set-up, as rttda_create is
    for the GPU); one sampled step is the oracle's sigma on those rows for
    every trajectory at the four RK4 stage times, and the full step is that
    time scaled by dim / nrows."""

    def __init__(self, mol, pulses, nrows: int):
        from oracle import rttda_oracle as orc
        self.orc = orc
        rng = np.random.default_rng(1)
        self.rows = np.sort(rng.choice(NDIM, size=min(nrows, NDIM), replace=False))
        hm = host_rows_molecule(mol, self.rows)
        self.A = orc.A_rows(hm, CX, self.rows)
        self.pulses, self.M, mcache = [], [], {}
        for p in pulses:
            d = tuple(float(x) for x in p["direction"])
            if d not in mcache:
                u = np.asarray(d) / np.linalg.norm(d)
                mcache[d] = orc.M_rows(*orc.dipole_along(hm, u), self.rows)
            self.M.append(mcache[d])
            self.pulses.append(orc.Pulse(kind=p["kind"], E0=p["E0"], omega=p.get("omega", 0.0),
                                         t0=p.get("t0", 0.0), fwhm=p.get("fwhm", 1.0),
                                         duration=p.get("duration", 0.0), direction=d))
        self.c = [rng.standard_normal(NDIM) + 1j * rng.standard_normal(NDIM) for _ in pulses]
        self.t = 0.0

    def step(self):
        for k, p in enumerate(self.pulses):
            c = self.c[k]
            for cs in (0.0, 0.5, 0.5, 1.0):
                sg = self.orc.sigma(self.A, self.M[k], self.orc.field(p, self.t + cs * DT), c)
                c[self.rows] = c[self.rows] + (-1j * DT) * sg * 1e-6
        self.t += DT

    def scale(self) -> float:
        return NDIM / len(self.rows)

    def save(self, path: str) -> None:
        np.savez(path, rows=self.rows, A=self.A, M=np.stack(self.M), c=np.stack(self.c),
                 pulses=json.dumps([p.__dict__ for p in self.pulses]))

    @classmethod
    def load(cls, path: str) -> "OracleSample":
        from oracle import rttda_oracle as orc
        z = np.load(path)
        s = cls.__new__(cls)
        s.orc, s.rows, s.A, s.t = orc, z["rows"], z["A"], 0.0
        s.M, s.c = list(z["M"]), list(z["c"])
        s.pulses = [orc.Pulse(**{k: (tuple(v) if isinstance(v, list) else v) for k, v in p.items()})
                    for p in json.loads(str(z["pulses"]))]
        return s


def sample_rows() -> int:
    """Rows of the oracle sample: a few seconds of CPU work per sampled step."""
    return {"fieldscan": 24, "large": 8}.get(NAME, 256)


def blas_threads() -> int:
    """Threads the oracle's BLAS runs on: threadpoolctl's count when it is
    installed, else the CPUs this process may use (OpenBLAS's default)."""
    for var in ("OPENBLAS_NUM_THREADS", "OMP_NUM_THREADS"):
        if os.environ.get(var, "").isdigit():
            return int(os.environ[var])
    try:
        from threadpoolctl import threadpool_info
        n = [i.get("num_threads", 1) for i in threadpool_info() if i.get("user_api") == "blas"]
        if n:
            return max(n)
    except Exception:
        pass
    try:
        return len(os.sched_getaffinity(0))
    except Exception:
        return os.cpu_count() or 1


def time_oracle(sample: OracleSample, nsteps: int, warmup: int = 1) -> dict:
    """Trajectory-steps/s of the oracle on its row sample, in this process
    (its BLAS on all cores unless the environment limits it)."""
    for _ in range(warmup):
        sample.step()
    t0 = time.perf_counter()
    for _ in range(nsteps):
        sample.step()
    dt_sample = (time.perf_counter() - t0) / nsteps
    T = len(sample.pulses)
    full_step = dt_sample * sample.scale()
    return {"value": T / full_step, "unit": UNIT, "cores": blas_threads(), "kind": "oracle",
            "sample": (f"oracle sigma on {len(sample.rows)} of {NDIM} rows of the explicit A and M_d (rows drawn "
                       f"with a fixed seed), {T} trajectories x 4 sigma per RK4 step, {nsteps} sampled steps, "
                       f"scaled x{sample.scale():.1f} to a full step; building the rows excluded as set-up"),
            "ms_per_step": full_step * 1e3}


def time_oracle_one_core(sample: OracleSample, nsteps: int) -> dict:
    """The same timing in a child process whose BLAS is limited to one thread
    (the thread count of a loaded BLAS cannot be changed from numpy)."""
    import tempfile
    with tempfile.TemporaryDirectory() as d:
        path = os.path.join(d, "sample.npz")
        sample.save(path)
        env = dict(os.environ, OMP_NUM_THREADS="1", OPENBLAS_NUM_THREADS="1", MKL_NUM_THREADS="1")
        out = subprocess.run([sys.executable, os.path.abspath(__file__), "--time-oracle-sample", path,
                              "--cpu-steps", str(nsteps), "--workload", NAME, "--naux", str(NAUX)],
                             env=env, capture_output=True, text=True, timeout=900)
        if out.returncode != 0:
            return {"error": out.stderr[-500:]}
        return json.loads(out.stdout.strip().splitlines()[-1])


def reference_pulses(mol):
    """The workload's pulses for the oracle arm.  The field scan's carrier
    frequency is set from the lowest orbital-energy gap here: the oracle
    cannot diagonalise A at this size, and the frequency does not change the
    cost of its sigma."""
    if NAME != "fieldscan":
        return workload_pulses(NAME)
    eo, ev = mol["eps_occ"], mol["eps_virt"]
    gap = float(ev.min() - eo.max()) if not hasattr(ev, "is_cuda") else float((ev.min() - eo.max()).item())
    return workload_pulses(NAME, gap)


def run_reference(args):
    rank, world, _ = dist_info()
    if rank != 0:
        return 0
    device = False
    if NAME in DEVICE_FACTORS:
        try:
            import torch
            device = torch.cuda.is_available()
        except Exception:
            device = False
    mol = make_molecule(NAME, device)
    pulses = reference_pulses(mol)
    sample = OracleSample(mol, pulses, sample_rows())
    del mol
    base = time_oracle(sample, args.steps, warmup=args.warmup)
    T = len(pulses)
    line = {"metric": METRIC, "value": base["value"], "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": base["ms_per_step"], "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": base_config("fp64 (CPU oracle)", 1, T), "impl": "reference",
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
        cmd = ["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits", "-lms", "100"]
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

TRAFFIC_FILE = os.path.join(ROOT, "profiles", "dram_traffic.txt")


def profiled_traffic(prec: str, cls: str, plan: dict):
    """DRAM bytes (dram__bytes_read.sum + dram__bytes_write.sum) per sigma
    build of a kernel class's main kernel, from the committed ncu summary
    table profiles/dram_traffic.txt, for this workload, precision and plan;
    None when the table has no capture of exactly this kernel and plan."""
    if not os.path.exists(TRAFFIC_FILE) or plan.get("z_chunk") != NAUX:
        return None  # the table's captures are of the unchunked exchange
    want = [NAME, str(NAUX), prec, cls, str(plan.get("main_kernel")), str(plan.get("main_bn")),
            str(plan.get("main_mb")), str(plan.get("main_kb")), str(plan.get("main_splits")),
            str(plan.get("main_cluster")), str(plan.get("main_grid"))]
    for line in open(TRAFFIC_FILE):
        f = line.split("#", 1)[0].split()
        if len(f) >= 13 and f[:11] == want:
            return {"bytes": float(f[11]), "source": f"profiles/{f[12]}"}
    return None


def algorithmic_work(prec: str, cls: str, T: int):
    """(method flop, hardware flop, bytes) of one sigma build's launches of a
    kernel class.

    exchange_main: K_(col,i),a = sum_{P,b} Z^P_(col,i),b B^P_ab with
    M = 2T nocc, N = nvirt, K = naux nvirt: the method's flop are 2MNK (one
    product, the P o v^2 C multiply-adds of the exchange); the hardware
    executes nprod products of the precision's hi/lo split; bytes = Z and
    B_vv read once (all planes)."""
    pi = PREC_INFO[prec]
    C = 2 * T
    o, v, P = NOCC, NVIRT, NAUX
    if cls == "exchange_main":
        M, N, K = C * o, v, P * v
        eb = 2 if pi["tensor"] else pi["fb"]
        zp = pi.get("zplanes", pi["planes"])
        f = 2.0 * M * N * K
        return f, pi["nprod"] * f, eb * (zp * M * K + pi["planes"] * P * v * v)
    if cls == "coulomb":
        f = 2 * 2.0 * P * o * v * C
        return f, f, 2.0 * P * o * v * (pi["fb"] if prec != "bf16x3" else 4)
    if cls == "exchange_z" and prec == "fp64oz":
        nz = P * o * v * C
        f = 2.0 * P * o * o * v * C
        return f, pi["nprod"] * f, (8 + 8 + 2 * 6) * nz + 2 * 6 * (P * o * o + o * v * C)
    if cls == "exchange_z":
        eb = 2 if pi["tensor"] else pi["fb"]
        zp = pi.get("zplanes", pi["planes"])
        nz = 3 if prec in ("bf16x3", "bf16x2") else pi["nprod"]
        f = 2.0 * P * o * o * v * C
        return f, nz * f, eb * (zp * P * o * v * C + pi["planes"] * P * o * o)
    return None, None, None


def roofline(prec: str, cls: str, prof_entry, T: int, peaks: dict, nsigma: int, plan: dict) -> dict:
    """Roofline of one kernel class.  The unit is one sigma build (one RK4
    stage): when the exchange is chunked over P, a stage is several launches
    of the class, so work and time are both taken per stage (the sum over
    its launches), which keeps achieved = work / duration for any chunking.

    achieved counts the method's flop (one product).  A tensor-bound class
    is set against the sustained (power-capped) bf16 peak: its kernels are
    timed inside steps of a seconds-long region, under the same power cap
    and clocks as the sustained measurement.  The fraction of the burst
    peak and the hardware rate (every product of the split) are beside it."""
    ms, n = prof_entry
    flop, hw_flop, byts = algorithmic_work(prec, cls, T)
    hbm = peaks.get("hbm_gbs", 6400.0)
    bf16_burst = peaks.get("bf16_tflops", 1800.0)
    bf16_sus = peaks.get("bf16_tflops_sustained", 1400.0)
    out = {"kernel": cls, "unit_of_work": "one sigma build (all launches of the class in one RK4 stage)",
           "avg_launch_ms": ms / max(n, 1), "launches_timed": n, "sigma_builds_timed": nsigma,
           "launches_per_sigma": n / max(nsigma, 1), "ms_per_sigma": ms / max(nsigma, 1), "traffic": None,
           "flop_per_sigma": flop, "hardware_flop_per_sigma": hw_flop, "bytes_per_sigma": byts}
    if flop is None or n == 0:
        out.update({"bound": None, "achieved": None, "peak": None, "unit": None, "frac": None})
        return out
    sec = ms / nsigma / 1e3
    pi = PREC_INFO[prec]
    if pi["tensor"]:
        cpeak, cunit, cbound = bf16_sus, "TFLOP/s", "tensor"
        csrc = ("of measured: bf16 sustained (MEASURED_PEAKS.json bf16_tflops_sustained; the class is timed "
                "inside a long step, under the power cap)")
    else:
        lanes = 128 if prec == "fp32" else 2
        cpeak = 148 * lanes * 2 * 2.032e9 / 1e12
        cunit, cbound = "TFLOP/s", "alu"
        csrc = (f"derived: 148 SM x {lanes} {'FP32' if prec == 'fp32' else 'FP64'} FMA/clk x 2 x 2032 MHz")
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
        out["frac_of_burst"] = flop / sec / 1e12 / bf16_burst
        out["hardware_tflops"] = hw_flop / sec / 1e12
    tr = profiled_traffic(prec, cls, plan)
    if tr is not None:
        # the table holds the captured kernel's bytes per sigma build (one
        # launch per stage with the exchange unchunked); the class's other
        # launches (the BF16 amplitude planes before the Z build) are not
        # counted
        out["traffic"] = tr["bytes"]
        out["traffic_source"] = tr["source"] + " (ncu dram__bytes_read.sum + dram__bytes_write.sum, this plan)"
        out["traffic_over_algorithmic"] = out["traffic"] / byts
    return out


# ---------------------------------------------------------------------------
# GPU arm
# ---------------------------------------------------------------------------
ACC_STEPS = 20     # horizon of the accuracy probe against the FP64-accurate path
ACC_STATES = 4     # lowest excitation energies compared (spectral peak positions)


def davidson(rb, prop, k, tol, max_iter=200):
    w, _, it = prop.eigenstates(k, tol=tol, max_iter=max_iter, allow_unconverged=True)
    return np.asarray(w), it


def kick_probe(rb, prop, nsteps):
    """Dipole and norm traces of one z-kicked trajectory (kappa = 1e-3) on
    the handle's molecule, for accuracy comparisons."""
    prop.set_field([dict(kind=rb.KICK, E0=KAPPA, direction=(0.0, 0.0, 1.0))])
    _, dip, nrm = prop.propagate(DT, nsteps, want_state=False)
    return dip[0], nrm[0]


def run_gpu(args):
    import torch
    rank, world, local = dist_info()
    torch.cuda.set_device(local)
    ranks = Ranks("nccl", "cuda")
    from paper_2601_16949_b300 import binding as rb
    barrier, max_over_ranks = ranks.barrier, ranks.max
    dev = torch.device("cuda", local)

    mol = make_molecule(NAME, NAME in DEVICE_FACTORS)
    wl_info = {}
    accuracy = None
    ref = None
    if not (args.no_accuracy or args.only_timed):
        # FP64-accurate reference (Ozaki digits on the tensor cores): the
        # lowest excitation energies by Davidson (the positions of the
        # lowest spectral peaks) and a kicked probe trajectory
        t0 = time.perf_counter()
        poz = rb.Propagator(mol, CX, "fp64oz")
        poz.set_field([dict(kind=rb.KICK, E0=KAPPA, direction=(0.0, 0.0, 1.0))] * 2)
        w_oz, it_oz = davidson(rb, poz, ACC_STATES, 1e-8)
        d_oz, n_oz = kick_probe(rb, poz, args.acc_steps)
        poz.close()
        ref = {"w": w_oz, "it": it_oz, "dip": d_oz, "nrm": n_oz, "s": time.perf_counter() - t0}
    if NAME == "fieldscan":
        if args.lambda_min > 0.0:
            lam, src = args.lambda_min, "given on the command line"
        elif ref is not None:
            lam = float(ref["w"][0])
            src = "Davidson on the FP64-accurate (Ozaki-digit) sigma build"
        else:
            p3 = rb.Propagator(mol, CX, "bf16x3")
            p3.set_field([dict(kind=rb.KICK, E0=KAPPA, direction=(0.0, 0.0, 1.0))] * 2)
            lam = float(davidson(rb, p3, 1, 1e-6)[0][0])
            p3.close()
            src = "Davidson on the BF16X3 sigma build"
        wl_info = {"lambda_min": lam, "lambda_min_source": src}
        pulses = workload_pulses(NAME, lam)
    else:
        pulses = workload_pulses(NAME)
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
    # per-kernel timing pass (events around every kernel class, same workload)
    rb.rttda_profile(h, True)
    kp = min(K, 40)
    pd_, pn_ = torch.zeros((T, kp + 1), dtype=torch.float64, device=dev), torch.zeros((T, kp + 1), dtype=torch.float64, device=dev)
    propagate(kp, pd_, pn_)
    torch.cuda.synchronize()
    prof = rb.rttda_profile_read(h)
    rb.rttda_profile(h, False)

    if args.only_timed:
        if rank == 0:
            print(json.dumps({"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": K,
                              "warmup": W, "ms_per_step": ms / K, "mode": "only-timed", "prec": args.prec,
                              "workload": NAME, "naux": NAUX, "plan": plan, "clocks": clk.summary(),
                              "class_ms_per_step": {k: round(v[0] / kp, 4) for k, v in prof.items()}}), flush=True)
        prop.close()
        ranks.close()
        return 0

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

    # accuracy of this precision against the FP64-accurate reference:
    # lowest excitation energies and the kicked probe (same handle, new batch)
    if ref is not None:
        tol = {"bf16": 1e-3, "bf16x2": 1e-5}.get(args.prec, 1e-7)
        w_p, it_p = davidson(rb, prop, ACC_STATES, tol)
        d_p, n_p = kick_probe(rb, prop, args.acc_steps)
        dd = ref["dip"] - ref["dip"][0]
        accuracy = {
            "reference": "fp64oz (FP64-accurate Ozaki-digit sigma build on the same molecule)",
            "peak_shift_ha": float(np.max(np.abs(w_p - ref["w"]))),
            "peak_shift_method": (f"lowest {ACC_STATES} excitation energies (the positions of the lowest spectral "
                                  "peaks of a kicked spectrum) by Davidson on each precision's own sigma build"),
            "excitation_energies_ha": w_p.tolist(), "reference_excitation_energies_ha": ref["w"].tolist(),
            "davidson_iterations": [int(it_p), int(ref["it"])],
            "norm_drift": float(np.max(np.abs(n_p - ref["nrm"]))),
            "dipole_rel_err": float(np.max(np.abs(d_p - ref["dip"])) / max(np.max(np.abs(dd)), 1e-300)),
            "probe": f"z kick kappa={KAPPA} from |0>, {args.acc_steps} RK4 steps of {DT} au (truncated horizon)",
            "gates": {"peak_shift_ha": 1e-4, "norm_drift": 1e-6},
            "reference_seconds": ref["s"]}
        accuracy["passes_gates"] = bool(accuracy["peak_shift_ha"] <= 1e-4 and accuracy["norm_drift"] <= 1e-6)
    prop.close()

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
    p64.close()

    # roofline of the dominant kernel class
    peaks = json.load(open(PEAKS_FILE)) if os.path.exists(PEAKS_FILE) else {}
    ms_cls = {k: v[0] for k, v in prof.items()}
    dom = max(ms_cls, key=ms_cls.get)
    # sigma builds in the profiled call: 4 per RK4 step; 2 per split-operator
    # step plus the call's first half step
    nsig = 4 * kp if args.integrator == "rk4" else 2 * kp + 1
    roof = roofline(args.prec, dom, prof[dom], T, peaks, nsig, plan)
    roof["class_ms_share"] = {k: round(v / max(sum(ms_cls.values()), 1e-30), 4) for k, v in ms_cls.items()}
    roof["class_ms_per_step"] = {k: round(v / kp, 4) for k, v in ms_cls.items()}
    roof["classes"] = {k: roofline(args.prec, k, prof[k], T, peaks, nsig, plan)
                       for k in ("coulomb", "exchange_z") if k in prof and prof[k][1] > 0}
    for k in list(roof["classes"]):
        roof["classes"][k] = {kk: roof["classes"][k].get(kk) for kk in
                              ("bound", "achieved", "peak", "unit", "frac", "ms_per_sigma", "traffic",
                               "traffic_over_algorithmic")}

    cpu = None
    if rank == 0 and not args.no_cpu_baseline:
        sample = OracleSample(mol, pulses, sample_rows())
        allc = time_oracle(sample, args.cpu_steps, warmup=1)
        one = time_oracle_one_core(sample, args.cpu_steps)
        cpu = {k: allc[k] for k in ("value", "unit", "cores", "kind", "sample")}
        cpu["single_core"] = {k: one.get(k) for k in ("value", "cores", "error") if k in one}
        cpu["host_cpus"] = os.cpu_count()

    dtype = {"fp64": "f64", "fp32": "f32", "bf16": "bf16", "bf16x3": "bf16x3", "bf16x2": "bf16x2",
             "fp64oz": "f64 (exchange: Ozaki BF16 digits)"}[args.prec]
    cfg = base_config(args.prec, world, T)
    if pop_info:
        cfg["populations"] = pop_info
    elif args.autocorrelation:
        cfg["autocorrelation"] = "recorded at every step, inside the timed region"
    cfg["integrator"] = {"rk4": "classical RK4 (4 sigma builds per step)",
                         "sso": "symplectic split operator (2 sigma builds per step)"}[args.integrator]
    cfg["factors"] = ("drawn on the GPU (seeded Philox)" if NAME in DEVICE_FACTORS else "drawn on the host (seeded PCG64)")
    cfg.update(wl_info)
    cfg.update({"fp64_path_traj_steps_per_s": fp64_rate, "speedup_vs_fp64_path": value / world / fp64_rate,
                "fp64_path": f"plain FP64, one trajectory (the batch's last), {k64} timed steps",
                "launches_per_step": per_step, "plan": plan})
    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": K, "warmup": W,
            "ms_per_step": ms / K, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": dtype, "data": "synthetic", "config": cfg, "accuracy": accuracy, "roofline": roof,
            "cpu_baseline": cpu, "e2e": e2e, "gpu_launches": int(launches1 - launches0), "clocks": clk.summary()}
    if rank == 0:
        print(json.dumps(line), flush=True)
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
    """Continuous-batching trace: Poisson arrivals, a random molecule, pulse
    and length per request, admitted by footprint; reports p50/p99
    time-to-spectrum and trajectory-steps/s.

    sizes "full" draws the serving workload's molecules (nocc U[16,192],
    nvirt U[64,1024] with nvirt >= 4 nocc, naux = 4 nvirt) with factors drawn
    on the GPU and handed to the server as device arrays (host FP64 factors
    of the largest would take 34 GB each); sizes "small" draws nocc U[16,48],
    nvirt U[64,192] on the host.  Device factors of a request exist from its
    arrival until the server admits it; to bound that memory the trace keeps
    at most --serving-pending such requests waiting in the server, later
    arrivals wait on the host, and their time to spectrum counts from the
    arrival."""
    import torch
    from paper_2601_16949_b300 import binding as rb
    from paper_2601_16949_b300 import synth
    torch.cuda.set_device(0)
    rng = np.random.default_rng(args.serving_seed)
    n = args.serving_requests
    full = args.serving_sizes == "full"
    arrivals = np.cumsum(rng.exponential(1.0 / args.serving_rate, n))
    spec = dict(gamma=1e-3, wmin=0.1, wmax=3.0, nfreq=512)
    shapes = []
    for k in range(n):
        while True:
            o = int(rng.integers(16, 193 if full else 49))
            v = int(rng.integers(64, 1025 if full else 193))
            if v >= 4 * o:
                break
        steps = int(rng.integers(args.serving_steps_min, args.serving_steps_max + 1))
        if rng.random() < 0.5:
            pulse = dict(kind=rb.KICK, E0=1e-3, direction=(0.0, 0.0, 1.0))
        else:
            pulse = dict(kind=rb.SIN2, E0=float(np.exp(rng.uniform(np.log(1e-3), np.log(5e-2)))),
                         omega=float(rng.uniform(0.4, 2.5)), duration=0.8 * steps * DT, direction=(0.0, 0.0, 1.0))
        shapes.append((o, v, 4 * v, steps, pulse))

    # The server's threads capture step graphs while this thread draws the
    # next molecules, so this thread synchronises only its own stream: a
    # device-wide synchronisation (or a cudaFree that implies one) would
    # invalidate a capture in flight, and the library would then run that
    # chunk without its graph.
    gen = torch.cuda.Stream()

    def make(k):
        o, v, P, steps, pulse = shapes[k]
        if not full:
            mol = synth.molecule(o, v, P, seed=1000 + k)
        else:
            with torch.cuda.stream(gen):
                mol = synth.molecule_device(o, v, P, seed=1000 + k)
            gen.synchronize()
        return rb.make_request(mol, CX, args.prec, pulse, DT, steps, **spec), mol

    # small molecules are drawn before the clock starts (host numpy takes up
    # to half a second each); the large ones on the GPU at arrival
    pre = None if full else [make(k) for k in range(n)]
    srv = rb.rttda_server_create(int(args.serving_budget_gb * (1 << 30)), args.serving_slots, args.serving_chunk)
    rb.rttda_server_set_grouping(srv, args.serving_grouping)
    ids, sub_t = [None] * n, [0.0] * n
    held = {}   # request index -> its device molecule, until admitted
    t0 = time.perf_counter()
    nxt = 0
    while nxt < n or held:
        now = time.perf_counter() - t0
        # release the device factors of admitted requests
        for k in list(held):
            if rb.rttda_server_poll(srv, ids[k])[0] != rb.REQ_PENDING:
                del held[k]
        while nxt < n and arrivals[nxt] <= now and (not full or len(held) < args.serving_pending):
            (q, mol) = make(nxt) if full else pre[nxt]
            ids[nxt] = rb.rttda_server_submit(srv, q)
            sub_t[nxt] = time.perf_counter() - t0
            if full:
                held[nxt] = (q, mol)
            nxt += 1
        time.sleep(0.005)
    for rid in ids:
        rb.rttda_server_wait(srv, rid, 7200.0)
    wall = time.perf_counter() - t0
    st = rb.rttda_server_stats_get(srv)
    polls = [rb.rttda_server_poll(srv, rid) for rid in ids]
    rb.rttda_server_destroy(srv)
    # time to spectrum from the arrival: host wait before submission plus
    # the server's submit -> spectrum time
    tts = np.array([(sub_t[k] - arrivals[k]) + polls[k][4] for k in range(n) if polls[k][0] == rb.REQ_DONE])
    line = {"mode": "serving", "metric": "time-to-spectrum p50/p99 and trajectory-steps/s (continuous batching)",
            "requests": n, "arrival_rate_per_s": args.serving_rate, "precision": args.prec,
            "grouping": {0: "off", 1: "by work", 2: "every eligible request"}[args.serving_grouping],
            "workload": (("serving workload sizes: nocc U[16,192], nvirt U[64,1024] with nvirt >= 4 nocc, naux = 4 nvirt, "
                          "factors drawn on the GPU" if full else
                          "small molecules: nocc U[16,48], nvirt U[64,192] with nvirt >= 4 nocc, naux = 4 nvirt") +
                         f"; kick or sin^2 pulse (E0 log-uniform 1e-3..5e-2); {args.serving_steps_min}-"
                         f"{args.serving_steps_max} RK4 steps of {DT} au"),
            "completed": st["completed"], "failed": st["failed"],
            "all_done": all(p[0] == rb.REQ_DONE for p in polls),
            "p50_time_to_spectrum_s": float(np.percentile(tts, 50)) if len(tts) else None,
            "p99_time_to_spectrum_s": float(np.percentile(tts, 99)) if len(tts) else None,
            "mean_time_to_spectrum_s": float(np.mean(tts)) if len(tts) else None,
            "server_p50_submit_to_spectrum_s": st["p50_latency_s"], "server_p99_submit_to_spectrum_s": st["p99_latency_s"],
            "trajectory_steps_per_s": st["trajectory_steps"] / max(st["busy_seconds"], 1e-9),
            "trajectory_steps": st["trajectory_steps"], "busy_seconds": st["busy_seconds"], "wall_seconds": wall,
            "max_concurrent": st["max_concurrent"], "grouped_requests": st["grouped"], "slots": args.serving_slots,
            "budget_gb": args.serving_budget_gb, "chunk_steps": args.serving_chunk}
    print(json.dumps(line), flush=True)
    return 0


def run_group_probe(args):
    """Throughput of S identical small requests submitted at once (kick,
    BF16), served with the grouped step and with one handle each: the
    launch-bound regime the grouped step is for."""
    import torch
    from paper_2601_16949_b300 import binding as rb
    from paper_2601_16949_b300 import synth
    torch.cuda.set_device(0)
    spec = dict(gamma=1e-3, wmin=0.1, wmax=3.0, nfreq=256)
    out = []
    for (o, v) in ((16, 64), (32, 128), (48, 192)):
        P = 4 * v
        for S in (1, 16):
            reqs = [rb.make_request(synth.molecule(o, v, P, seed=2000 + k), CX, "bf16",
                                    dict(kind=rb.KICK, E0=KAPPA, direction=(0.0, 0.0, 1.0)), DT,
                                    args.probe_steps, **spec) for k in range(S)]
            for g in (1, 0):
                srv = rb.rttda_server_create(64 << 30, S, args.probe_steps)
                rb.rttda_server_set_grouping(srv, 2 if g else 0)
                t0 = time.perf_counter()
                ids = [rb.rttda_server_submit(srv, q) for q in reqs]
                for rid in ids:
                    rb.rttda_server_wait(srv, rid, 600.0)
                wall = time.perf_counter() - t0
                st = rb.rttda_server_stats_get(srv)
                rb.rttda_server_destroy(srv)
                out.append({"nocc": o, "nvirt": v, "naux": P, "requests": S, "grouping": g,
                            "steps_per_request": args.probe_steps, "completed": st["completed"],
                            "traj_steps_per_s": st["trajectory_steps"] / wall, "wall_s": wall,
                            "us_per_step_per_request": wall / args.probe_steps * 1e6 / S})
                print(json.dumps(out[-1]), flush=True)
    return 0


def main():
    ap = argparse.ArgumentParser(description=__doc__)
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="fieldscan", choices=sorted(WORKLOADS))
    ap.add_argument("--prec", default="bf16", choices=["fp64", "fp32", "bf16", "bf16x3", "bf16x2", "fp64oz"])
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
    ap.add_argument("--group-probe", action="store_true",
                    help="throughput of identical small requests, grouped step against one handle each")
    ap.add_argument("--probe-steps", type=int, default=1000)
    ap.add_argument("--serving-sizes", default="small", choices=["small", "full"])
    ap.add_argument("--serving-steps-min", type=int, default=200)
    ap.add_argument("--serving-steps-max", type=int, default=2000)
    ap.add_argument("--serving-grouping", type=int, default=1, choices=(0, 1, 2),
                    help="grouped step of small BF16 requests: 0 off, 1 by work (default), 2 every eligible request")
    ap.add_argument("--serving-pending", type=int, default=2,
                    help="full sizes: most requests with device factors waiting in the server")
    ap.add_argument("--fp64-steps", type=int, default=2)
    ap.add_argument("--e2e-steps", type=int, default=10)
    ap.add_argument("--cpu-steps", type=int, default=3)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-accuracy", action="store_true",
                    help="skip the accuracy leg against the FP64-accurate (Ozaki-digit) path")
    ap.add_argument("--acc-steps", type=int, default=ACC_STEPS,
                    help="RK4 steps of the kicked accuracy probe")
    ap.add_argument("--time-oracle-sample", default="", help=argparse.SUPPRESS)
    ap.add_argument("--lambda-min", type=float, default=0.0,
                    help="field scan: use this lambda_min(A) instead of solving for it (profiler captures)")
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
    if args.time_oracle_sample:
        r = time_oracle(OracleSample.load(args.time_oracle_sample), args.cpu_steps, warmup=0)
        print(json.dumps(r), flush=True)
        return 0
    if args.impl == "reference":
        return run_reference(args)
    if args.accuracy:
        return run_accuracy(args)
    if args.serving:
        return run_serving(args)
    if args.group_probe:
        return run_group_probe(args)
    return run_gpu(args)


if __name__ == "__main__":
    sys.exit(main())
