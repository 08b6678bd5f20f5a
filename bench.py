"""Benchmark of the CHYM GB300 simulator.

Default workload ("n100", one bench step): the Moebius ladder N=100 (ring bonds
-1 plus antipodal rungs -1) and an SK +-1 N=100 instance, each at hyperspin
dimension D in {2 (XY machine, no annealing), 3, 4} with 4096 runs = 32 pump
values x 128 replicas, 20000 Euler-Maruyama steps (dt = 0.01; D >= 3 anneal
linearly over the second half), then the Ising readout, energies and
ground-state statistics.  Other workloads (--workload): "sk1000" (SK +-1 and
Gaussian N=1000, D=4, 16384 runs, 50000 steps) and "sk800" (SK +-1 N=800, D=4,
65536 runs, 50000 steps), which run on the large-N tensor-core path, and "uneven"
(512 SK +-1 instances, N uniform in [50, 2000], D in {2,3,4,8}, 64 runs each over
16 pumps, 30000 steps) as one batch whose planner costs are tuned on the device.

Metric: hyperspin-steps/s (N * D * runs * steps per second) and ground-state
hits per second.  Beside the mixed-precision form the line carries the plain
FP32 form of the same workload and, for the default workload, the mixed form
with the learned early exit in continuous operation (finished and retired runs
reseeded), each with its ground-state hits per second.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--workload n100|sk1000|sk800]
  python bench.py --impl reference ...   # the FP64 CPU oracle on the host cores

Multi-GPU (torchrun): every rank runs its own replica of the workload with its
own seeds (runs are independent, no collective on the data path); value = all
ranks' work / max rank time.
"""
import argparse
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time
from dataclasses import dataclass, field

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "GS hits/s and hyperspin-steps/s (N·D·runs·steps), mixed+learned vs plain FP32"
UNIT = "hyperspin-steps/s"
EPS_HAT = 0.5
INSTANCE_SEED = 0xC0FFEE
PEAK_FALLBACK = {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "bf16_tflops_sustained": 1700.0}


@dataclass
class Workload:
    key: str
    title: str
    graphs: list            # (name, kind, N)
    D: tuple
    n_h: int
    reps: int
    steps: int
    compare_plain: bool = True
    learned: bool = False
    notes: dict = field(default_factory=dict)

    @property
    def runs(self):
        return self.n_h * self.reps


WORKLOADS = {
    "n100": Workload("n100", "moebius N=100 + SK+-1 N=100, D in {2,3,4}, 4096 runs/graph "
                     "(32 h x 128 replicas), 20000 steps dt=0.01",
                     [("moebius", "moebius", 100), ("sk", "sk", 100)], (2, 3, 4), 32, 128, 20000,
                     learned=True),
    "sk1000": Workload("sk1000", "SK+-1 and Gaussian N(0,1/N) N=1000, D=4, 16384 runs "
                       "(32 h x 512 replicas), 50000 steps dt=0.01",
                       [("sk", "sk", 1000), ("gauss", "gauss", 1000)], (4,), 32, 512, 50000,
                       compare_plain=False),
    "sk800": Workload("sk800", "SK+-1 N=800, D=4, 65536 runs (32 h x 2048 replicas), "
                      "50000 steps dt=0.01",
                      [("sk", "sk", 800)], (4,), 32, 2048, 50000, compare_plain=False),
    "uneven": Workload("uneven", "512 SK+-1 instances, N uniform in [50, 2000], D uniform in "
                       "{2,3,4,8}, 64 runs each (16 h x 4 replicas), 30000 steps dt=0.01, "
                       "one tuned batch", [], (2, 3, 4, 8), 16, 4, 30000, compare_plain=False),
    "fig4": Workload("fig4", "size scaling of Fig. 4: 20 % sparse +-1 graphs, N = 10..100, 16 graphs "
                     "per N; CIM (D=1, 51 h) and CHYM+DA (D=2 annealed, 21 h), 32 replicas, "
                     "20000 steps dt=0.01", [], (1, 2), 21, 32, 20000, compare_plain=False),
    "sparse": Workload("sparse", "Moebius ladders N=2048 and N=4096, D=3, 2048 runs each "
                       "(32 h x 64 replicas), 20000 steps dt=0.01: coupling over the nonzeros of J",
                       [("moebius", "moebius", 2048), ("moebius4k", "moebius", 4096)], (3,), 32, 64, 20000,
                       compare_plain=False),
    "sk20_fp64": Workload("sk20_fp64", "SK+-1 N=20, D=3, 256 runs (8 h x 32 replicas), 3000 steps "
                          "dt=0.01 (1500 + 1500 annealing), FP64 oracle-comparison mode",
                          [("sk", "sk", 20)], (3,), 8, 32, 3000, compare_plain=False),
    "map": Workload("map", "SK+-1 N=100, D=3, the cavity round-trip map of Eq. 1-2 (a=0.95, d=0.1, "
                    "beta=100), 32 gain values K = K_th (1 + dK), dK in [0, 0.25], 512 replicas "
                    "each (16384 runs), 20000 round trips", [("sk", "sk", 100)], (3,), 32, 512, 20000,
                    compare_plain=False),
}
MAP_CAVITY = {"a": 0.95, "d": 0.1, "beta": 100.0}
MAP_GAIN_SPAN = 0.25
FIG4_NS = tuple(range(10, 101, 10))
FIG4_GRAPHS = 16
UNEVEN_INSTANCES = 512


def workload_specs(w, rank):
    """Every context of a workload: name, graph kind, N, D, instance seed (or None),
    pump values, replicas and the machine constants (gamma, kappa, schedule kind)."""
    def spec(name, kind, N, D, seed, n_h=None, gamma=25.0, mode=None):
        kappa, skind = mode if mode else mode_for(D)
        return {"name": name, "kind": kind, "N": N, "D": D, "seed": seed,
                "n_h": n_h or w.n_h, "reps": w.reps, "gamma": gamma, "kappa": kappa, "skind": skind}
    if w.key == "uneven":
        from paper_2308_02329_gb300 import inputs
        comp = inputs.uneven_instances(UNEVEN_INSTANCES, INSTANCE_SEED + 4)
        return [spec(f"sk{N}_{i}", "sk", N, D, seed + 1000003 * rank)
                for i, (N, D, seed) in enumerate(comp)]
    if w.key == "fig4":
        from paper_2308_02329_gb300 import scaling
        out = []
        for N, g, seed in scaling.graph_set(FIG4_NS, FIG4_GRAPHS, seed=0x5CA1E + 7 * rank):
            for mode, m in scaling.MODES.items():
                out.append(spec(f"sparse{N}_{g}", "sparse", N, m["D"], seed,
                                n_h=51 if m["D"] == 1 else 21, gamma=m["gamma"],
                                mode=(m["kappa"], 1 if m["anneal"] else 0)))
                out[-1]["mode"] = mode
        return out
    if w.key == "map":   # one context per gain value: eps and gamma follow the gain
        out = []
        for dk in np.linspace(0.0, MAP_GAIN_SPAN, w.n_h):
            for name, kind, N in w.graphs:
                for D in w.D:
                    out.append(spec(name, kind, N, D, None, n_h=1, mode=(0.0, 0)))
                    out[-1]["gain_rel"] = float(dk)
        return out
    return [spec(name, kind, N, D, None) for name, kind, N in w.graphs for D in w.D]


def build_graph(kind, N, rank, seed=None):
    from paper_2308_02329_gb300 import inputs
    if kind == "moebius":
        return inputs.mobius_ladder(N)
    if kind == "sparse":
        return inputs.sparse_pm1(N, 0.2, seed)
    if kind == "er1":
        return inputs.sparse_pm1(N, 0.01, seed if seed is not None else INSTANCE_SEED + 3 + 1000 * rank)
    if kind == "sk":
        return inputs.sk_pm1(N, seed if seed is not None else INSTANCE_SEED + 1 + 1000 * rank)
    return inputs.gaussian(N, INSTANCE_SEED + 2 + 1000 * rank)


def mode_for(D):
    """D = 2: XY machine without annealing (kappa L = 1e-3); D >= 3: annealing mode
    (kappa L = 0.1); beta b^2 = 25 in both."""
    if D == 2:
        return 1e-3, 0
    return 0.1, 1


def workload_config(w, prec_name, sim_steps):
    if w.graphs:
        graphs = [f"{n}_{N}" for n, _, N in w.graphs]
    elif w.key == "fig4":
        graphs = [f"{FIG4_GRAPHS} sparse +-1 graphs (density 0.2) per N in {list(FIG4_NS)}"]
    else:
        graphs = [f"{UNEVEN_INSTANCES} SK+-1 instances, N in [50, 2000]"]
    cfg = {"workload": w.title, "key": w.key, "graphs": graphs, "D": list(w.D),
           "runs_per_graph": w.runs, "n_h": w.n_h, "replicas": w.reps, "steps": sim_steps,
           "precision": prec_name, "l2": "flushed between steps (256 MiB write)"}
    if w.key == "map":
        cfg["cavity"] = dict(MAP_CAVITY)
        cfg["gains"] = f"K_th (1 + dK), dK = linspace(0, {MAP_GAIN_SPAN}, {w.n_h}), one context each"
    return cfg


def map_euler(lam, gain_rel):
    """Euler form of one round trip (dt = 1) at gain K = K_th (1 + gain_rel), from the
    package's reduction of the map: the (dt, sigma, init_std, gamma, kappa, eps) tuple
    and the pump value h."""
    from paper_2308_02329_gb300.round_trip import Cavity
    cav = Cavity(**MAP_CAVITY)
    prm, h = cav.euler((1.0 + gain_rel) * cav.threshold(lam), sigma=1e-3, init_std=0.1)
    return (prm.dt, prm.sigma, prm.init_std, prm.gamma, prm.kappa, prm.eps), h


def measured_peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as fh:
            d = json.load(fh)
        return d, "measured"
    except (OSError, ValueError):
        return dict(PEAK_FALLBACK), "fallback"


def alu_ops_per_element(D, nnz_row, coupling_on_alu, wide_mul_ops=2):
    """Algorithmic ALU lane-operations per element-step (one x_{p,mu} advanced once).

    Noise: one Philox4x32-10 block per four normals (per spin and 4 components for D >= 3,
    per 4/D spins for D <= 2): 10 rounds x [2 products of 32 x 32 -> 64 bits + 2 three-input
    xors + 2 key adds].  A 64-bit product is two 32-bit results (high and low word), each an
    integer multiply, which the SM issues on its FMA-heavy pipe at half the FP32 FMA rate:
    it counts wide_mul_ops = 2 lane-operations (1 gives the unweighted count), so a block
    is 80 (60).  Box-Muller 12 ops per pair (2 int->float, 2 scalings, log, radius scaling,
    sqrt, angle, sin, cos, 2 products).  Drift + Euler-Maruyama update: 6.5 ops (norm
    share, x^2, cubic/loss FMA, product, coupling FMA, noise add).  Coupling on the ALU
    adds nnz_row FMAs (dense J: N)."""
    if D <= 2:      # the 4/D spins of a Philox block share it (all four normals used)
        blocks_per_el, pairs_per_el = 0.25, 0.5
    else:
        blocks_per_el, pairs_per_el = -(-D // 4) / D, -(-D // 2) / D
    ops = 10.0 * (2 * wide_mul_ops + 4) * blocks_per_el + 12.0 * pairs_per_el + 6.5
    if coupling_on_alu:
        ops += nnz_row
    return ops


FP64_NOMINAL_TFLOPS = 1.25   # GB300 FP64 rate (nominal; no measured figure on this machine)


def step_roofline(jobs, prec, steps_total, dur, clock_info, peaks, peak_src, prec_name):
    """Roofline object of the step kernels of one timed region (dur: their span, s).

    Large-N tensor-core contexts: algorithmic 2 N^2 D flops per run and step and the
    issued products (K padded to 128, two BF16 products for +-1 J, three for real J)
    against the sustained dense BF16 peak.  FP64 mode: the FP64 flops of the coupling
    (2 N) and of the drift and update (10) per element against the nominal FP64 rate (the
    noise's FP64 log and sine are not counted).  Otherwise the ALU lane-operations of
    alu_ops_per_element against 152 SMs x 128 FP32 lanes at the median SM clock."""
    from paper_2308_02329_gb300 import chym
    tc = prec in (chym.PREC_BF16X2, chym.PREC_FP8)
    large = any(j["N"] > 128 and not j["ctx"].uses_csr(prec) for j in jobs) and tc
    if large:
        alg = steps_total * sum(2.0 * j["N"] ** 2 * j["D"] * j["runs"] for j in jobs)
        # issued products: BF16 J x_hi, then J x_lo in BF16 (or in e4m3 at twice the rate in
        # FP8 mode with +-1 J), plus J_lo x_hi for real J; in BF16-equivalent flops
        bf16_eq, fp8 = 0.0, 0.0
        for j in jobs:
            f = 2.0 * (128 * -(-j["N"] // 128)) ** 2 * j["D"] * j["runs"] * steps_total
            if j["name"] == "gauss":
                bf16_eq += 3 * f
            elif prec == chym.PREC_FP8:
                bf16_eq += f + 0.5 * f
                fp8 += f
            else:
                bf16_eq += 2 * f
        peak = peaks["bf16_tflops_sustained"] * 1e12
        out = {"bound": "tensor", "achieved": alg / dur / 1e12, "peak": peak / 1e12,
               "unit": "TFLOP/s", "frac": alg / dur / peak, "traffic": None,
               "issued_tflops": bf16_eq / dur / 1e12, "issued_frac": bf16_eq / dur / peak,
               "kernel": "large-N tcgen05 step (BF16 hi + " +
                         ("e4m3 lo for +-1 J" if prec == chym.PREC_FP8 else "BF16 lo") + ", FP32 accumulate)",
               "peak_note": f"dense BF16 sustained, {peak_src}; FP8 products counted at half their flops "
                            "(the e4m3 rate is twice the BF16 rate)"}
        if fp8:
            out["issued_fp8_tflops"] = fp8 / dur / 1e12
        return out
    if prec == chym.PREC_FP64:
        alg = steps_total * sum((2.0 * j["N"] + 10.0) * j["N"] * j["D"] * j["runs"] for j in jobs)
        peak = FP64_NOMINAL_TFLOPS * 1e12
        return {"bound": "fp64", "achieved": alg / dur / 1e12, "peak": peak / 1e12,
                "unit": "TFLOP/s", "frac": alg / dur / peak, "traffic": None,
                "kernel": "SIMT step kernel (FP64)",
                "peak_note": "nominal FP64 rate of the part (of nominal, not measured); "
                             "coupling and update flops only, the noise transform uncounted"}
    on_alu = prec == chym.PREC_FP32

    def ops(wide):
        return steps_total * sum(
            alu_ops_per_element(j["D"], j["N"] if j["name"] in ("sk", "gauss") else j["nnz"],
                                on_alu or j["ctx"].uses_csr(prec), wide) *
            j["N"] * j["D"] * j["runs"] for j in jobs)
    alg, alg1 = ops(2), ops(1)
    sm_mhz = clock_info.get("sm_mhz") or peaks.get("sm_max_mhz", 2070.0)
    peak = 152 * 128 * sm_mhz * 1e6
    return {"bound": "alu", "achieved": alg / dur / 1e12, "peak": peak / 1e12,
            "unit": "Tlane-op/s", "frac": alg / dur / peak, "traffic": None,
            "frac_unweighted": alg1 / dur / peak,
            "kernel": ("SIMT step kernel, coupling over the nonzeros of J (FP32)"
                       if all(j["ctx"].uses_csr(prec) for j in jobs) else
                       "SIMT step kernels (FP32)" if on_alu else "chym step kernel (" + prec_name + ")"),
            "peak_note": "152 SMs x 128 FP32 lanes x median SM clock during the region; a 32-bit "
                         "integer multiply counts 2 (half-rate pipe), frac_unweighted counts it 1"}


# DRAM bytes (read + write) of the dominant kernel per launch, from ncu captures of these
# kernels as they stand (dram__bytes_read.sum + dram__bytes_write.sum), by workload and
# precision: None where no capture of the current kernel exists.
TRAFFIC = {
    ("n100", "bf16x2"): (3.25e7, "the three step_tc_kernel launches of one bench step (D = 2, 3, 4; "
                                 "7.5 + 10.8 + 14.2 MB read, writes stay in L2)"),
    ("sk800", "fp8"): (2.972e9, "one step_k2_kernel launch (one integration step): 1486 MB captured "
                                "on 32768 runs, doubled for 65536 (traffic grows with the columns)"),
}

REPLAY_RUNS, REPLAY_STEPS = 64, 400


def replay_against_oracle(jobs, steps):
    """64 runs of each context (every (runs/64)-th run, so every pump) replayed from their
    seeds in a fresh context for `steps` steps on the GPU and on the FP64 oracle: the largest
    state error relative to its own (run, component) scale, and the share of runs whose Ising
    energies agree exactly."""
    import oracle.oracle as O
    from paper_2308_02329_gb300 import chym, inputs
    out = {}
    for j in jobs:
        pick = np.linspace(0, j["runs"] - 1, REPLAY_RUNS).astype(int)
        reps = j["runs"] // j["n_h"]
        h_run = inputs.h_per_run(j["h"], reps)[pick]
        seeds = np.ascontiguousarray(j["seeds"][pick])
        J = j["J"]
        ctx = chym.Context(J, j["D"], chym.J_REAL if j["name"] == "gauss" else chym.J_PM1)
        sch = chym.Schedule(j["sched"].kind, j["sched"].k_anneal, j["sched"].k_total)
        # one pump per replayed run: REPLAY_RUNS pump values, one replica each
        ctx.run(j["prm"], h_run, seeds, steps, sch)
        X, _ = ctx.get_state()
        E = ctx.energy()
        ctx.close()
        t0 = time.perf_counter()
        p = j["prm"]
        Xo = O.run(J, j["D"], h_run, seeds,
                   O.Params(dt=p.dt, sigma=p.sigma, init_std=p.init_std, gamma=p.gamma, kappa=p.kappa,
                            eps=p.eps), O.Schedule(sch.kind, sch.k_anneal, sch.k_total), steps)
        el = time.perf_counter() - t0
        Eo = O.ising_energies(J, O.readout(Xo))
        glob = float(np.max(np.abs(Xo)))
        scale = np.maximum(np.max(np.abs(Xo), axis=1, keepdims=True), 1e-12 * glob)
        err = np.max(np.abs(X - Xo) / scale, axis=(1, 2))
        # exact integers for +-1 couplings; FP64 sums in another order for real J
        same = (E == Eo) if j["name"] != "gauss" else np.isclose(E, Eo, rtol=1e-12, atol=1e-12)
        out[j["name"]] = {"runs": REPLAY_RUNS, "steps": steps, "of_steps": j["sched"].k_total,
                          "state_rel_err_max": float(err.max()),
                          "state_rel_err_median": float(np.median(err)),
                          "energy_equal_frac": float(np.mean(same)),
                          "oracle_seconds": el}
    return out


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled every 200 ms in the background."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.path = None

    def start(self):
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except OSError:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        rows = []
        with open(self.path) as fh:
            for line in fh:
                parts = [p.strip() for p in line.split(",")]
                if len(parts) >= 9:
                    rows.append(parts)
        os.unlink(self.path)
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}

        def num(v):
            try:
                return float(v)
            except ValueError:
                return None
        sm = [num(r[1]) for r in rows if num(r[1]) is not None]
        mx = [num(r[2]) for r in rows if num(r[2]) is not None]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in rows for i in range(4) if r[5 + i] == "Active"})
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(mx) if mx else None, "reasons": reasons,
                "samples": len(rows)}


def merge_over_ranks(elapsed, hits, dist, device):
    """Whole-job view of one timed region: the slowest rank's time (max) and the
    ground-state hits of all ranks (sum).  Each rank integrates its own replica of
    the workload, so there is no exchange on the data path; this is the only
    collective, once per timed region."""
    import torch
    t = torch.tensor([float(elapsed)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    h = torch.tensor([float(hits)], dtype=torch.float64, device=device)
    dist.all_reduce(h, op=dist.ReduceOp.SUM)
    return float(t.item()), int(h.item())


def oracle_jobs(w):
    """(J, D, oracle params, oracle schedule) of every (graph, D) of a workload; for the
    uneven workload, of every 32nd instance (a bounded sample)."""
    import oracle.oracle as O
    jobs = []
    specs = workload_specs(w, 0)
    if w.key in ("uneven", "fig4"):
        specs = specs[::32]
    elif w.key == "map":
        specs = specs[::8]
    cache = {}
    for sp in specs:
        kind, N, seed = sp["kind"], sp["N"], sp["seed"]
        if (kind, N, seed) not in cache:
            J = build_graph(kind, N, 0, seed)
            lam = float(np.linalg.eigvalsh(J)[-1])
            cache[(kind, N, seed)] = (J, lam if lam > 0 else 1.0)
        J, lam = cache[(kind, N, seed)]
        if "gain_rel" in sp:
            (dt, sg, i0, ga, ka, ep), h = map_euler(lam, sp["gain_rel"])
            prm = O.Params(dt=dt, sigma=sg, init_std=i0, gamma=ga, kappa=ka, eps=ep)
            jobs.append((J, sp["D"], prm, O.Schedule(0, 0, 0), h))
            continue
        prm = O.Params(dt=0.01, sigma=1e-3, init_std=0.1, gamma=sp["gamma"], kappa=sp["kappa"],
                       eps=EPS_HAT / lam)
        jobs.append((J, sp["D"], prm, O.Schedule(sp["skind"], w.steps // 2, w.steps), None))
    return jobs


def time_oracle(jobs, runs, steps, threads):
    """Wall time of the FP64 oracle: every job, `runs` runs x `steps` steps + energies."""
    import oracle.oracle as O
    from paper_2308_02329_gb300 import inputs
    t0 = time.perf_counter()
    for J, D, prm, sch, h_map in jobs:
        N = J.shape[0]
        seeds = inputs.run_seeds(INSTANCE_SEED, runs)
        h = np.resize(inputs.pump_grid(1.0 - EPS_HAT, 8), runs) if h_map is None else np.full(runs, h_map)
        X = O.init_state(N, D, seeds, prm.init_std)
        O.integrate(J, X, h, seeds, prm, sch, 0, steps, threads=threads)
        O.ising_energies(J, O.readout(X))
    return time.perf_counter() - t0


def cpu_baseline_sample(w, target_s=10.0):
    """The FP64 oracle on a bounded sample of the same workload, on all host cores."""
    threads = os.cpu_count()
    jobs = oracle_jobs(w)
    runs = max(2 * threads, 16)
    probe = 20
    t = time_oracle(jobs, runs, probe, threads)
    steps = int(max(probe, min(w.steps, probe * target_s / max(t, 1e-6))))
    el = time_oracle(jobs, runs, steps, threads)
    work = sum(J.shape[0] * D * runs * steps for J, D, *_ in jobs)
    return {"value": work / el, "unit": UNIT, "cores": threads, "kind": "oracle",
            "sample": f"{len(jobs)} (graph, D) contexts of the workload, {runs} runs x {steps} of "
                      f"{w.steps} steps each, FP64, OpenMP over runs; {el:.1f} s"}


def run_reference(args, w, rank, world):
    """The FP64 CPU oracle as it stands, timed on the host cores on this workload."""
    if rank != 0:
        return 0
    threads = os.cpu_count()
    jobs = oracle_jobs(w)
    runs = max(threads, 16)
    per_step_target = 6.0
    t = time_oracle(jobs, runs, 20, threads)
    steps = int(max(20, min(w.steps, 20 * per_step_target / max(t, 1e-6))))
    for _ in range(args.warmup):
        time_oracle(jobs, runs, steps, threads)
    el = sum(time_oracle(jobs, runs, steps, threads) for _ in range(args.steps))
    work = sum(J.shape[0] * D * runs * steps for J, D, *_ in jobs)
    value = work * args.steps / el
    sample = (f"per step: {len(jobs)} (graph, D) contexts of the workload, {runs} runs x {steps} of {w.steps} "
              f"steps each, FP64, OpenMP over runs")
    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * el / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": workload_config(w, "fp64 (CPU oracle)", w.steps),
            "impl": "reference",
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": threads, "kind": "oracle",
                             "sample": sample},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


def pack_jobs(jobs, lams, graphs, prec, torch):
    """Fig. 4 graphs of each machine mode packed into contexts of up to 128 spins (blocks
    of a block-diagonal J; each graph keeps eps_i = eps_hat / lambda_max(J_i) through the
    per-spin coupling weights, so all share the pump grid).  A pack job reads its
    graphs' energies as segments."""
    from paper_2308_02329_gb300 import chym, packing
    by_mode = {}
    for j, lam in zip(jobs, lams):
        by_mode.setdefault(j["mode"], []).append((j, lam))
    out = []
    for mode, items in by_mode.items():
        for k, members in enumerate(packing.plan([j["N"] for j, _ in items])):
            P = packing.build([graphs[items[i][0]["name"]] for i in members], list(range(len(members))))
            j0 = items[members[0]][0]
            ctx = chym.Context(P.J, j0["D"])
            lam = [items[i][1] for i in members]
            if len(members) > 1:
                ctx.set_coupling_weights(packing.spin_weights(P, [1.0 / l if l > 0 else 0.0 for l in lam]))
            eps = EPS_HAT if len(members) > 1 else (EPS_HAT / lam[0] if lam[0] > 0 else 0.0)
            prm = chym.Params(dt=0.01, sigma=1e-3, init_std=0.1, gamma=j0["gamma"], kappa=j0["kappa"],
                              eps=eps, prec=prec)
            out.append(dict(j0, name=f"pack{k}_{mode}", N=P.N, ctx=ctx, prm=prm, seg=P.seg_begin,
                            members=[items[i][0]["name"] for i in members],
                            nnz=max(1, int((P.J != 0).sum(1).mean()))))
        for j, _ in items:
            j["ctx"].close()
    return out


def pack_hits(j, gs, sp):
    """Ground-state hits of a pack job's graphs, from their segment energies."""
    Eseg = j["ctx"].energy_segments(j["seg"], sp)
    return sum(int(np.sum(Eseg[:, b] == gs[m])) for b, m in enumerate(j["members"])), Eseg


def learned_leg(jobs, w, sim_steps, gs, batch, stream, chunks, plain, train_batches=1, burn_in=10):
    """Mixed precision + learned early exit on the same contexts.

    Setup (untimed): every context generates labelled trajectories with its own fresh
    seeds (features at 10 % of the schedule, outcome at the end), one network is
    trained on all of them on the GPU, and each context gets its own retire
    threshold, set for a 10 % false-negative rate on half of its held-out runs (no
    retirement where that half holds fewer than 5 successes); the other half
    measures the false-negative rate.  Timed: continuous operation (every slot
    always busy, finished and retired slots reseeded) of all contexts as one batch
    for `chunks` chunks of 10 % of the schedule, with and without the network, after
    10 uncounted burn-in chunks (one schedule length) that spread the slots over
    their schedules.  A context keeps its threshold only where its held-out test
    half predicts a gain of more than 5 % (early_exit.expected_gain); elsewhere the
    network is not consulted.  Returns the leg's JSON object."""
    import torch
    from paper_2308_02329_gb300 import chym
    from paper_2308_02329_gb300 import early_exit as EE
    from paper_2308_02329_gb300 import inputs
    K, k_dec = sim_steps, sim_steps // 10
    sp = stream.cuda_stream
    Fs, Es, Fv, Ev = [], [], [], []
    t_setup = time.perf_counter()
    for i, j in enumerate(jobs):
        F, E = [], []
        for tb in range(train_batches):
            f, _, e = EE.generate(j["ctx"], j["prm"], j["sched"], j["h"],
                                  inputs.run_seeds(0x5EED0000 + i + 0x100 * tb, w.runs), K, k_dec,
                                  gs[j["name"]], sp)
            F.append(f)
            E.append(e)
        Fs.append(torch.cat(F))
        Es.append(np.concatenate(E))
        f, _, e = EE.generate(j["ctx"], j["prm"], j["sched"], j["h"],
                              inputs.run_seeds(0x7A1D0000 + i, w.runs), K, k_dec, gs[j["name"]], sp)
        Fv.append(f)
        Ev.append(e)
    # success = ending at the reference energy: the exact or best-known ground state, lowered
    # to the best energy any of these runs reached (for instances without an exact one)
    e_ref = {}
    for i, j in enumerate(jobs):
        low = float(min(np.nanmin(Es[i]), np.nanmin(Ev[i])))
        e_ref[i] = gs[j["name"]] = min(gs[j["name"]], low)

    def label(E, i):
        return torch.from_numpy((np.abs(E - e_ref[i]) <= 1e-9 * max(1.0, abs(e_ref[i]))).astype(np.float32)).cuda()
    ys = [label(Es[i], i) for i in range(len(jobs))]
    yv = [label(Ev[i], i) for i in range(len(jobs))]
    F, y = torch.cat(Fs), torch.cat(ys)
    net = chym.MLP(seed=4, max_batch=1024)
    loss = EE.train(net, F, y, epochs=30, batch=512, lr=2e-3, stream=sp)
    rng = np.random.default_rng(0)
    thetas, per_ctx = [], []
    fn_num = fn_den = 0
    for i, j in enumerate(jobs):
        sv = EE.logits(net, Fv[i], sp).cpu().numpy()
        yvn = yv[i].cpu().numpy()
        perm = rng.permutation(len(sv))
        cal, tst = perm[: len(sv) // 2], perm[len(sv) // 2:]
        pos = yvn[tst] > 0.5
        th, gain, fn_i, rho_i = -np.inf, None, None, None
        if int((yvn[cal] > 0.5).sum()) >= 5 and int(pos.sum()) >= 5:
            th = EE.threshold_for_fn(sv[cal], yvn[cal], 0.1)
            fn_i = float(np.mean(sv[tst][pos] < th))
            rho_i = float(np.mean(sv[tst] < th))
            gain = EE.expected_gain(fn_i, rho_i, k_dec / K)
            if gain <= 1.05:
                th = -np.inf
        if np.isfinite(th):
            fn_num += int((sv[tst][pos] < th).sum())
            fn_den += int(pos.sum())
        thetas.append(th)
        per_ctx.append({"context": f'{j["name"]}_D{j["D"]}', "p_success": float(yvn.mean()),
                        "e_ref": e_ref[i], "positives_train": int(ys[i].sum().item()),
                        "positives_heldout": int((yvn > 0.5).sum()),
                        "fn_test": fn_i, "retire_frac_test": rho_i, "expected_gain": gain,
                        "exit_enabled": bool(np.isfinite(th)),
                        "theta": None if not np.isfinite(th) else float(th)})
    setup_s = time.perf_counter() - t_setup
    if not any(np.isfinite(t) for t in thetas):
        # no context has enough successes to set a threshold: the network is never
        # consulted, so continuous operation with it equals operation without it
        net.close()
        out = {"gs_hits_per_s": None, "gain_vs_mixed": None, "exit_enabled": False,
               "fn_rate_heldout": None, "fn_target": 0.1, "positives_heldout": fn_den,
               "per_context": per_ctx, "train_rows": int(F.shape[0]), "train_loss": loss,
               "setup_s": setup_s,
               "note": "too few successful runs to set a retire threshold (at least 5 in each "
                       "held-out half are required): no false-negative rate is quoted and the "
                       "exit stays off; the learned form is the mixed form here (gain 1)"}
        return out

    def run(with_net, key):
        streams = [EE.SeedStream(key + i) for i in range(len(jobs))]
        return EE.continuous_many([j["ctx"] for j in jobs], [j["prm"] for j in jobs],
                                  [j["sched"] for j in jobs], [j["h"] for j in jobs],
                                  [w.runs] * len(jobs), streams, K, k_dec,
                                  [gs[j["name"]] for j in jobs], chunks,
                                  net if with_net else None, thetas, sp, batch=batch,
                                  burn_in=burn_in)
    mixed = run(False, 0xC0A7)
    learned = run(True, 0xC0A7)
    net.close()
    out = {"gs_hits_per_s": learned.hits_per_second,
           "mixed_continuous_gs_hits_per_s": mixed.hits_per_second,
           "gain_vs_mixed": learned.hits_per_second / mixed.hits_per_second
           if mixed.hits_per_second > 0 else None,
           "hits_per_mstep": {"learned": learned.hits_per_mstep, "mixed": mixed.hits_per_mstep},
           "completed": {"learned": learned.completed, "mixed": mixed.completed},
           "retired": learned.retired, "seconds": {"learned": learned.seconds,
                                                   "mixed": mixed.seconds},
           "integrate_seconds": {"learned": learned.integrate_seconds,
                                 "mixed": mixed.integrate_seconds},
           "p_success_completed": {"learned": learned.hits / max(learned.completed, 1),
                                   "mixed": mixed.hits / max(mixed.completed, 1)},
           "fn_rate_heldout": fn_num / fn_den if fn_den else None, "fn_target": 0.1,
           "positives_heldout": fn_den, "per_context": per_ctx,
           "train_rows": int(F.shape[0]), "train_loss": loss, "setup_s": setup_s,
           "window": f"{chunks} chunks of {k_dec} steps after {burn_in} uncounted burn-in chunks "
                     f"(decision at 10 % of {K})"}
    if out["gain_vs_mixed"] is not None and out["gain_vs_mixed"] <= 1.0:
        out["note"] = "the learned exit does not pay on this workload: gain_vs_mixed <= 1"
    if plain and plain["gs_hits_per_s"] > 0:
        out["ratio_vs_plain_fp32"] = learned.hits_per_second / plain["gs_hits_per_s"]
    return out


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="chym", choices=["chym", "reference"])
    ap.add_argument("--workload", default="n100", choices=sorted(WORKLOADS))
    ap.add_argument("--prec", default="bf16x2", choices=["bf16x2", "fp8", "fp32", "fp64"])
    ap.add_argument("--no-compare-plain", dest="compare_plain", action="store_false")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-learned", action="store_true")
    ap.add_argument("--no-pack", action="store_true",
                    help="fig4: one context per graph instead of graphs packed into 128-spin contexts")
    ap.add_argument("--no-tune", action="store_true",
                    help="keep the planner's default cost model instead of measuring it")
    ap.add_argument("--learned", action="store_true",
                    help="run the learned early-exit leg on this workload too")
    ap.add_argument("--learned-train-batches", type=int, default=1,
                    help="learned leg: batches of the workload's runs generated for training")
    ap.add_argument("--learned-burn-in", type=int, default=10,
                    help="learned leg: uncounted chunks before the timed window")
    ap.add_argument("--learned-chunks", type=int, default=30,
                    help="chunks of 10 %% of the schedule in the learned leg's timed window "
                         "(after 10 uncounted burn-in chunks)")
    ap.add_argument("--sim-steps", type=int, default=0,
                    help="integration steps per run (default: the workload's); for profiling")
    ap.add_argument("--replicas", type=int, default=0,
                    help="replicas per pump value (default: the workload's); for profiling")
    ap.add_argument("--no-configs", action="store_true",
                    help="default workload: skip the one-step lines of the other configurations")
    args = ap.parse_args()
    args.warmup = max(args.warmup, 3)
    w = WORKLOADS[args.workload]
    if args.replicas:
        w.reps = args.replicas
    sim_steps = args.sim_steps or w.steps

    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if args.impl == "reference":
        return run_reference(args, w, rank, world)

    import torch
    import torch.distributed as dist

    torch.cuda.set_device(local)
    if world > 1:
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    line = measure(args, w, sim_steps, rank, world, local)
    if line is not None and world == 1 and args.workload == "n100" and not args.no_configs:
        line["configs"] = {key: measure_config(args, key, rank, world, local) for key in EXTRA_CONFIGS}
    if line is not None:
        print(json.dumps(line), flush=True)
    if world > 1:
        dist.destroy_process_group()
    return 0


# One timed bench step of each of these, beside the default workload's line: the
# FP64 oracle-comparison mode on its SK N=20 case, the two large-N workloads at their
# full size (50000 steps each) and the uneven batch (30000 steps), with the precision
# each runs in (FP8 mode for +-1 couplings on the large-N path).
EXTRA_CONFIGS = {"sk20_fp64": "fp64", "sk1000": "fp8", "sk800": "fp8", "uneven": "fp8"}


def measure_config(args, key, rank, world, local):
    """One timed step of workload `key` at its full size after three short warm-up steps
    (WARM_STEPS integration steps each), with its own clocks, roofline, ground-state
    hits and CPU baseline; for sk1000 also the replay of 64 runs against the oracle."""
    sub = argparse.Namespace(**vars(args))
    sub.steps, sub.warmup = 1, 3
    sub.prec = EXTRA_CONFIGS[key]
    sub.compare_plain, sub.no_e2e, sub.no_learned = False, True, True
    w = WORKLOADS[key]
    line = measure(sub, w, w.steps, rank, world, local, warm_steps=min(w.steps, WARM_STEPS),
                   replay=key == "sk1000" and not args.no_cpu_baseline)
    keep = ("value", "unit", "ms_per_step", "steps", "warmup", "dtype", "config", "gs_hits_per_s",
            "e_gs", "roofline", "cpu_baseline", "clocks", "gpu_launches", "replay64", "tuning")
    out = {k: line[k] for k in keep if k in line}
    if len(out.get("e_gs", {})) > 8:   # the uneven batch: one reference per instance
        out["e_gs"] = {"instances": len(out["e_gs"]),
                       "note": "best energy of the warm-up and timed runs of each instance"}
    return out


WARM_STEPS = 1000


def measure(args, w, sim_steps, rank, world, local, warm_steps=None, replay=False):
    """Set up a workload's contexts, warm up, time args.steps bench steps and return the
    JSON line (rank 0; None on the other ranks).  warm_steps: integration steps of each
    warm-up step (default: the full sim_steps)."""
    import torch
    import torch.distributed as dist
    from paper_2308_02329_gb300 import chym, inputs

    dev = torch.device("cuda", local)
    stream = torch.cuda.current_stream(dev)
    prec = {"bf16x2": chym.PREC_BF16X2, "fp8": chym.PREC_FP8, "fp32": chym.PREC_FP32,
            "fp64": chym.PREC_FP64}[args.prec]

    # ---------------- setup (untimed): instances, references, device inputs ----------
    jobs, gs = [], {}
    graphs = {}
    for gi, sp in enumerate(workload_specs(w, rank)):
        name, kind, N, D, seed = sp["name"], sp["kind"], sp["N"], sp["D"], sp["seed"]
        if name not in graphs:
            J = build_graph(kind, N, rank, seed)
            graphs[name] = J
            jkind = chym.J_REAL if kind == "gauss" else chym.J_PM1
            if kind == "moebius":
                gs[name] = chym.ground_state_mobius(N)
            elif w.key == "uneven":
                gs[name] = float("inf")    # best energy of the warm-up runs (below)
            elif N <= 24:
                c1 = chym.Context(J, 1, jkind)
                gs[name] = c1.ground_state_exact()[0]
                c1.close()
            else:
                c1 = chym.Context(J, 1, jkind)
                restarts, sweeps = ((16, 1000) if kind == "sparse" else (64, 2000)) if N <= 200 else (4, 400)
                gs[name] = c1.ground_state_search(restarts=restarts, sweeps=sweeps, seed=11)[0]
                c1.close()
        J = graphs[name]
        jkind = chym.J_REAL if kind == "gauss" else chym.J_PM1
        ctx = chym.Context(J, D, jkind)
        n_h, runs = sp["n_h"], sp["n_h"] * sp["reps"]
        h = inputs.pump_grid(1.0 - EPS_HAT, n_h)
        sd = INSTANCE_SEED + 7919 * rank + 97 * gi + D if seed is None else seed + D
        seeds = inputs.run_seeds(sd, runs)
        jobs.append(dict(name=name, N=N, D=D, ctx=ctx, kappa=sp["kappa"], skind=sp["skind"],
                         J=J if replay else None,
                         gain_rel=sp.get("gain_rel"),
                         gamma=sp["gamma"], mode=sp.get("mode"), n_h=n_h, runs=runs, h=h,
                         seeds=seeds, d_h=torch.from_numpy(h).to(dev),
                         d_seeds=torch.from_numpy(seeds.view(np.int64)).to(dev),
                         d_E=torch.empty(runs, dtype=torch.float64, device=dev),
                         nnz=max(1, int((J != 0).sum(1).mean()))))
        if w.key == "uneven":
            del graphs[name]     # the context holds its own copy of J
    # lambda_max of every context (host Lanczos; ctypes releases the GIL)
    from concurrent.futures import ThreadPoolExecutor
    with ThreadPoolExecutor(max_workers=os.cpu_count() or 4) as pool:
        lams = list(pool.map(lambda j: j["ctx"].lambda_max(), jobs))
    for j, lam in zip(jobs, lams):
        j["prm"] = chym.Params(dt=0.01, sigma=1e-3, init_std=0.1, gamma=j["gamma"], kappa=j["kappa"],
                               eps=EPS_HAT / lam if lam > 0 else 0.0, prec=prec)
        j["sched"] = chym.Schedule(j["skind"], sim_steps // 2 if j["skind"] else 0, sim_steps)
        if j["gain_rel"] is not None:   # the round-trip map: dt = 1, per-gain constants
            (dt, sg, i0, ga, ka, ep), h = map_euler(lam, j["gain_rel"])
            j["prm"] = chym.Params(dt=dt, sigma=sg, init_std=i0, gamma=ga, kappa=ka, eps=ep, prec=prec)
            j["h"] = np.array([h])
            j["d_h"] = torch.from_numpy(j["h"]).to(dev)
    if w.key == "fig4" and not args.no_pack:
        jobs = pack_jobs(jobs, lams, graphs, prec, torch)
    graphs.clear()
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)
    streams = [torch.cuda.Stream(dev) for _ in jobs]
    batch = chym.Batch([j["ctx"] for j in jobs])
    spans = []
    # the planner's cost model, measured for this batch on this device (setup, untimed)
    for j in jobs:
        j["ctx"].run_device(j["prm"], j["d_h"].data_ptr(), j["n_h"], j["d_seeds"].data_ptr(),
                            j["runs"], 0, j["sched"], stream.cuda_stream)
    tuning = None
    if prec in (chym.PREC_BF16X2, chym.PREC_FP8) and not args.no_tune:
        tuning = batch.tune([j["prm"] for j in jobs], [j["sched"] for j in jobs],
                            probe_steps=min(256, sim_steps), stream=stream.cuda_stream)

    def one_step(record=False, steps=None):
        """init every (graph, D), integrate all of them together as one batch (persistent
        launches spread over all SMs) for `steps` (default: sim_steps) steps, energies
        and the ground-state statistics.  Device inputs.  Returns the ground-state hits
        of this step."""
        flush.fill_(1.0)
        sp = stream.cuda_stream
        for j in jobs:
            j["ctx"].run_device(j["prm"], j["d_h"].data_ptr(), j["n_h"], j["d_seeds"].data_ptr(),
                                j["runs"], 0, j["sched"], sp)
        e0 = torch.cuda.Event(enable_timing=record)
        e1 = torch.cuda.Event(enable_timing=record)
        e0.record(stream)
        batch.run([j["prm"] for j in jobs], [j["sched"] for j in jobs], steps or sim_steps, sp)
        e1.record(stream)
        for j in jobs:
            if "seg" not in j:
                j["ctx"].energy_device(j["d_E"].data_ptr(), 0, sp)
        hits = 0
        if record:
            spans.append((e0, [(e0, e1)]))
            for j in jobs:
                hits += pack_hits(j, gs, sp)[0] if "seg" in j else \
                    int(j["ctx"].stats(gs[j["name"]], 0, sp)["n_hits"])
        return hits

    def set_prec(pv):
        for j in jobs:
            j["prm"].prec = pv

    def timed_region(K):
        """Barrier, K bench steps bracketed by CUDA events, barrier; max over ranks."""
        spans.clear()
        if world > 1:
            dist.barrier()
        torch.cuda.synchronize()
        t0 = torch.cuda.Event(enable_timing=True)
        t1 = torch.cuda.Event(enable_timing=True)
        t0.record(stream)
        hits = 0
        for _ in range(K):
            hits += one_step(record=True)
        t1.record(stream)
        torch.cuda.synchronize()
        el = t0.elapsed_time(t1) / 1e3
        if world > 1:
            el, hits = merge_over_ranks(el, hits, dist, dev)
        return el, hits

    # warm-up; the references of non-exact instances also take the best energy found
    for _ in range(args.warmup):
        one_step(steps=warm_steps)
    torch.cuda.synchronize()
    for j in jobs:
        if "seg" in j:
            Eseg = pack_hits(j, gs, stream.cuda_stream)[1]
            for b, m in enumerate(j["members"]):
                if np.isfinite(Eseg[:, b]).any():
                    gs[m] = min(gs[m], float(np.nanmin(Eseg[:, b])))
        elif j["name"] != "moebius":
            gs[j["name"]] = min(gs[j["name"]], float(j["d_E"].min().item()))

    # ---------------- timed region: device-resident inputs ----------------
    clocks = ClockSampler(local)
    clocks.start()
    elapsed, hits_total = timed_region(args.steps)
    clock_info = clocks.stop()
    work_step = sum(j["N"] * j["D"] * j["runs"] * sim_steps for j in jobs)
    value = work_step * args.steps * world / elapsed
    if args.steps == 1 and world == 1 and w.key in ("sk1000", "sk800", "uneven"):
        # no exact ground state at these sizes: the reference is the best energy of the
        # search and of every run of the timed step, and its hits are counted against it
        hits_total = 0
        for j in jobs:
            E = j["d_E"].cpu().numpy()
            gs[j["name"]] = min(gs[j["name"]], float(np.nanmin(E)))
            hits_total += int(np.sum(np.abs(E - gs[j["name"]]) <= 1e-9 * max(1.0, abs(gs[j["name"]]))))

    # roofline of the dominant kernel (the step kernels of the batch, concurrent):
    # achieved = their algorithmic work / the span of the batched integration
    dur = 0.0
    for fork, marks in spans:
        starts = [fork.elapsed_time(e0) for e0, _ in marks]
        ends = [fork.elapsed_time(e1) for _, e1 in marks]
        dur += (max(ends) - min(starts)) / 1e3
    peaks, peak_src = measured_peaks()
    roofline = step_roofline(jobs, prec, args.steps * sim_steps, dur, clock_info, peaks, peak_src,
                             args.prec)
    if (w.key, args.prec) in TRAFFIC and sim_steps == w.steps and not args.replicas:
        roofline["traffic"], roofline["traffic_note"] = TRAFFIC[(w.key, args.prec)]

    # ---------------- the plain FP32 form on the same workload ----------------
    plain = None
    if args.compare_plain and w.compare_plain and prec != chym.PREC_FP32:
        set_prec(chym.PREC_FP32)
        one_step()
        el_p, hits_p = timed_region(args.steps)
        set_prec(prec)
        dur_p = 0.0
        for fork, marks in spans:
            dur_p += (max(fork.elapsed_time(e1) for _, e1 in marks) -
                      min(fork.elapsed_time(e0) for e0, _ in marks)) / 1e3
        plain = {"value": work_step * args.steps * world / el_p, "unit": UNIT,
                 "gs_hits_per_s": hits_p / el_p, "ms_per_step": 1e3 * el_p / args.steps,
                 "dtype": "f32", "form": "SIMT FP32 coupling product, same workload",
                 "roofline": step_roofline(jobs, chym.PREC_FP32, args.steps * sim_steps, dur_p,
                                           clock_info, peaks, peak_src, "fp32")}

    # ---------------- e2e: host inputs through the public API ----------------
    e2e = None
    if not args.no_e2e:
        pin_h = [torch.from_numpy(j["h"]).pin_memory() for j in jobs]
        pin_s = [torch.from_numpy(j["seeds"].view(np.int64)).pin_memory() for j in jobs]
        E_host = [torch.empty(j["runs"], dtype=torch.float64).pin_memory() for j in jobs]
        if world > 1:
            dist.barrier()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for _ in range(args.steps):
            flush.fill_(1.0)
            sp = stream.cuda_stream
            for j, ph, ps in zip(jobs, pin_h, pin_s):
                j["ctx"].run(j["prm"], ph.numpy(), ps.numpy().view(np.uint64), 0, j["sched"], sp)
            batch.run([j["prm"] for j in jobs], [j["sched"] for j in jobs], sim_steps, sp)
            for j, eh in zip(jobs, E_host):
                if "seg" in j:
                    pack_hits(j, gs, sp)
                    continue
                eh.copy_(torch.from_numpy(j["ctx"].energy(stream=sp)))
                j["ctx"].stats(gs[j["name"]], 0, sp)
        torch.cuda.synchronize()
        el2 = time.perf_counter() - t0
        if world > 1:
            el2, _ = merge_over_ranks(el2, 0, dist, dev)
        h2d = sum(j["n_h"] * 8 + j["runs"] * 8 for j in jobs)
        d2h = sum(j["runs"] * 8 * len(j["members"]) if "seg" in j else j["runs"] * 8 + 64 + j["n_h"] * 8
                  for j in jobs)
        e2e = {"value": work_step * args.steps * world / el2, "unit": UNIT,
               "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h}

    # ---------------- Fig. 4: size scaling of the success probability ----------------
    scaling_study = None
    if w.key == "fig4":
        from paper_2308_02329_gb300 import scaling
        rows = {}
        for j in jobs:   # figures of the last timed step's runs
            if "seg" in j:
                Eseg = pack_hits(j, gs, stream.cuda_stream)[1]
                per = [(m, scaling.figures(Eseg[:, b], gs[m], j["n_h"])) for b, m in enumerate(j["members"])]
            else:
                per = [(j["name"], j["ctx"].stats(gs[j["name"]], 0, stream.cuda_stream))]
            for m, st in per:
                Nm, g = int(m.split("_")[0][len("sparse"):]), int(m.split("_")[1])
                rows.setdefault(j["mode"], []).append(scaling.GraphResult(
                    Nm, g, float(gs[m]), Nm <= 24, float(st["P_max"]),
                    float(st["W_range"]), float(st["W_scan"]), float(st["dE_mean"])))
        scaling_study = {}
        for mode, rs in rows.items():
            agg = scaling.aggregate(rs)
            a, c, used = scaling.fit_exponential(list(agg), [agg[N]["P_max"]["mean"] for N in agg])
            scaling_study[mode] = {"decay_a": a, "decay_c": c, "fit_points": used,
                                   "P_max_mean": {str(N): agg[N]["P_max"]["mean"] for N in agg},
                                   "P_max_iqr": {str(N): [agg[N]["P_max"]["q25"], agg[N]["P_max"]["q75"]]
                                                 for N in agg},
                                   "W_range_mean": {str(N): agg[N]["W_range"]["mean"] for N in agg},
                                   "dE_mean": {str(N): agg[N]["dE_mean"]["mean"] for N in agg}}

    # ---------------- mixed + learned early exit (continuous operation) ----------------
    learned = None
    if (w.learned or args.learned) and not args.no_learned and world == 1 and \
            prec in (chym.PREC_BF16X2, chym.PREC_FP8):
        learned = learned_leg(jobs, w, sim_steps, gs, batch, stream, args.learned_chunks, plain,
                              args.learned_train_batches, args.learned_burn_in)

    if rank == 0:
        cpu = None
        if not args.no_cpu_baseline and world == 1:
            cpu = cpu_baseline_sample(w)
        # launches of our kernels per bench step: pump indices, init, energy and
        # statistics per context (a pack of graphs: pump indices, init and one segment
        # energy launch, its statistics are host-side); one persistent launch per
        # dimension for the small-N contexts; the large-N path adds 3 layout kernels per
        # context, one grouped GEMM launch per dimension and integration step, and one
        # step-counter kernel per 16-step graph; FP32/FP64 contexts and sparse ones take
        # one persistent SIMT launch each
        bf16 = prec in (chym.PREC_BF16X2, chym.PREC_FP8)
        small = [j for j in jobs if j["N"] <= 128 and bf16]
        large = [j for j in jobs if j["N"] > 128 and bf16 and not j["ctx"].uses_csr(prec)]
        sparse = [j for j in jobs if j["ctx"].uses_csr(prec)]
        per_step = sum(3 if "seg" in j else 4 for j in jobs) + len({j["D"] for j in small}) + \
            3 * len(large) + (sim_steps * len({j["D"] for j in large}) + sim_steps // 16 if large else 0) + (
                len(sparse) if bf16 else len(jobs))
        line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
                "steps": args.steps, "warmup": args.warmup,
                "ms_per_step": 1e3 * elapsed / args.steps, "higher_is_better": True,
                "scaling": "weak", "vs_baseline": None,
                "dtype": {chym.PREC_BF16X2: "bf16x2+f32", chym.PREC_FP8: "bf16+e4m3+f32",
                          chym.PREC_FP32: "f32"}.get(prec, "f64"),
                "data": "synthetic", "config": workload_config(w, args.prec, sim_steps),
                "gs_hits_per_s": hits_total / elapsed,
                "e_gs": {k: float(v) for k, v in gs.items()},
                "roofline": roofline, "cpu_baseline": cpu, "e2e": e2e, "clocks": clock_info,
                "plain_fp32": plain,
                "gs_hits_ratio_vs_plain": (hits_total / elapsed) / plain["gs_hits_per_s"]
                if plain and plain["gs_hits_per_s"] > 0 else None,
                "gpu_launches": args.steps * per_step}
        if tuning is not None:
            line["tuning"] = tuning
        if scaling_study is not None:
            line["scaling_study"] = scaling_study
        if w.key == "fig4":
            line["packing"] = None if args.no_pack else {
                "contexts": len(jobs), "graphs": sum(len(j["members"]) for j in jobs),
                "lanes_used": sum(j["N"] for j in jobs) / (128.0 * len(jobs)),
                "form": "graphs packed into contexts of up to 128 spins (block-diagonal J, "
                        "eps_i per graph through per-spin coupling weights)"}
        if learned is not None:
            line["learned"] = learned
            line["gs_hits_ratio_learned_vs_plain"] = learned.get("ratio_vs_plain_fp32")
        if replay:
            line["replay64"] = replay_against_oracle(jobs, REPLAY_STEPS)
    else:
        line = None
    batch.close()
    for j in jobs:
        j["ctx"].close()
    return line


if __name__ == "__main__":
    sys.exit(main())
