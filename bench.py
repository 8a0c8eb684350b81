#!/usr/bin/env python
"""Throughput of the compact finite-difference hot path on GB300.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--workload NAME] [--prec P] [--impl ours|reference]

One step = one pass of the whole path over one batch: ghost exchange of all
fields (matrix G, Eq. example_G), then all requested derivative ops of every
field on every MeshBlock (closed block systems, Eq. sch_cent_om, plus the
hybrid iteration, Eq. iter_center_P, on uniform meshes).  Metric: Gpoint-ops/s
= interior points x fields x ops / step time.  Prints ONE JSON line (rank 0).

Under torchrun (N > 1) every rank runs an independent replica of the workload
(the path has no data exchange between replicas), value = units of all
ranks / max-over-ranks time ("weak" scaling).  --impl reference times the
oracle on the host cores instead (rank 0 only).
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "Gpoint-ops/s: split-BF16 TC CFD vs FP64 banded solve, err ≤1e-6 vs FP64"
ADVECT_METRIC = "Gpoint-ops/s: upwinded shift advection (biased CCU X_2 pencil solves)"
ADV2D_METRIC = "Gpoint-ops/s: 2D advection, upwinded CCU X_2, 2S RK + KO"
L2_BYTES = 129 * 2 ** 20
FP64_NOMINAL_GFLOPS = 1250.0      # GB300 FP64 (non-tensor) nominal, profiling recipe table

PREC = {"fp64_banded": 0, "tc_bf16x3": 1, "tc_bf16_exact": 2, "tc_tf32": 3}


def arithmetic_name(prec: int, field_dtype: str) -> str:
    """The arithmetic a path computes in (the field dtype is only its input/output format)."""
    io = f"{field_dtype} in/out"
    return {0: f"f64 (banded solve), {io}",
            1: f"bf16 hi/lo split, 3 products, fp32 accumulate, {io}",
            2: f"bf16 digit slices, 15 exact-integer products in fp32, {io}",
            3: f"tf32, 1 product, fp32 accumulate, {io}"}[prec]

WORKLOADS = {
    # one periodic 32^3 block (no interfaces: the undecomposed cyclic scheme), one field (8 sine modes,
    # integer k in [1, 12]), d_x only with the 6th-order tridiagonal Pade P^1_2: launch-bound
    "cfd32_b32_f1_p12_dx": dict(kind="uniform", NM=32, N=32, nf=1, fields=1, dtype="f64", n_iter=0, scheme="P12",
                                ops="dx"),
    # 256^3 periodic, 512 blocks of 32^3, 4 FP64 fields, 9 ops, closed blocks (dense D = A^-1 B)
    "cfd256_b32_f4_fp64": dict(kind="uniform", NM=256, N=32, nf=4, fields=3, dtype="f64", n_iter=0),
    # 128^3 periodic, 512 blocks of 16^3, 4 FP64 fields, 9 ops
    "cfd128_b16_f4_fp64": dict(kind="uniform", NM=128, N=16, nf=4, fields=2, dtype="f64", n_iter=0),
    # 128^3 periodic, 64 blocks of 32^3, 4 FP64 fields: the small case for ncu captures
    "cfd128_b32_f4_fp64": dict(kind="uniform", NM=128, N=32, nf=4, fields=3, dtype="f64", n_iter=0),
    # 448 blocks 16^3 + 64 blocks 32^3, 22 FP32 fields, 9 ops, closures only
    "box448x16_64x32_f22_fp32": dict(kind="boxinbox", nf=22, fields=4, dtype="f32", n_iter=0),
    # linear wave u_tt = Laplacian u, 256^3 as 512 blocks of 32^3, plane waves |k| <= 20, RK4, dt = 0.25 dx
    "wave256_b32_rk4": dict(kind="wave", NM=256, N=32, nf=2, dtype="f64", n_iter=0, modes=8, kmax=20.0),
    # shifted wave (Eq. toyShiftWaveEqnSys, flat background) with a constant shift, 2S RK + Kreiss-Oliger,
    # upwinded CCU X_2 advective terms, 256^3 as 512 blocks of 32^3, same plane waves (exact solution
    # known: each mode's frequency is |k| - beta.k)
    "shiftwave256_b32_x2_lsrk": dict(kind="wave", NM=256, N=32, nf=2, dtype="f64", n_iter=1, modes=8, kmax=20.0,
                                     shift=(0.3, -0.2, 0.1)),
    # 2D advection u_t + c . grad u = 0 (Sec. "Two dimensional advection"): 192^2 as 12 x 12 blocks of 16^2
    # (one 16-point block thick in z), the paper's initial profile g(x) h(y), direction 30 degrees,
    # upwinded CCU X_2, one iteration, 2S RK + Kreiss-Oliger (sigma 0.04, r = 4), dt = dx / 10
    "adv2d192_b16_x2_lsrk": dict(kind="adv2d", NM=192, N=16, nf=1, dtype="f64", n_iter=1, angle_deg=30.0,
                                 cfl=0.1),
    # upwinded shift advection sum_i beta^i d_i f (Eq. biasderapproxadv) with the CCU X_2^-
    # scheme and its mirror (Tab. ccux_deg_one_col), 256^3 as 512 blocks of 32^3, 4 FP64 fields,
    # one iteration of Eq. iter_left_X
    "advect256_b32_x2_f4_fp64": dict(kind="advect", NM=256, N=32, nf=4, fields=3, dtype="f64", n_iter=1),
    # the same on 128^3 as 64 blocks of 32^3 (small case for ncu captures)
    "advect128_b32_x2_f4_fp64": dict(kind="advect", NM=128, N=32, nf=4, fields=3, dtype="f64", n_iter=1),
    # the shift-advection term of all 22 FP32 fields of the Z4c-shaped workload (448 blocks of 16^3 +
    # 64 of 32^3, analytic ghosts at the coarse/fine interfaces, closures only)
    "advect_box448x16_64x32_f22_fp32": dict(kind="advect", mesh="boxinbox", N=16, nf=22, fields=4, dtype="f32",
                                            n_iter=0),
}
DEFAULT_WORKLOAD = "cfd256_b32_f4_fp64"

# DRAM traffic of the dominant kernel per launch, from an ncu capture of the current kernel
# (dram__bytes_read.sum + dram__bytes_write.sum, averaged over the launches of one step), keyed
# by (workload, path, n_iter).  Values with their profile summary under profiles/.
MEASURED_TRAFFIC = {
    # 256^3 as 512 blocks of 32^3, 4 FP64 fields, 9 ops: one-pass capture of the 6 k_dense
    # launches of a step at full size (profiles/k_dense_tc_exact_cfd128_b32_f4.md)
    ("cfd256_b32_f4_fp64", "tc_bf16_exact", 0): 1757165301,
    # 448 x 16^3 + 64 x 32^3, 22 FP32 fields, 9 ops: one-pass capture of the 24 k_dense launches
    # of a step at full size (profiles/launches_box448x16_64x32_f22_fp32_tc_exact.md)
    ("box448x16_64x32_f22_fp32", "tc_bf16_exact", 0): 415090976,
}


def scheme_descs(name: str = "Q13"):
    """Tuned (Q^1_3[eta_c=1], Tabs. num_deg_one/two) interior schemes as the paper prints them,
    or the 6th-order Pade P^1_2 (Tabs. pade_deg_one/two) for name "P12".

    The closures are built by the library (C_0 matching, closure=NULL).
    """
    if name == "P12":
        d1 = {"deriv": 1, "order": 6, "a": 1.0 / 3.0, "rhs": [v / 36.0 for v in (-1.0, -28.0, 0.0, 28.0, 1.0)]}
        d2 = {"deriv": 2, "order": 6, "a": 2.0 / 11.0, "rhs": [v / 44.0 for v in (3.0, 48.0, -102.0, 48.0, 3.0)]}
        return d1, d2
    d1 = {"deriv": 1, "order": 6, "a": 0.37987923,
          "rhs": [0.0023272948, -0.052602255, -0.78165660, 0.0, 0.78165660, 0.052602255, -0.0023272948]}
    d2 = {"deriv": 2, "order": 6, "a": 0.24246603,
          "rhs": [-0.0037062571, 0.14095923, 0.95445144, -2.1834088, 0.95445144, 0.14095923, -0.0037062571]}
    return d1, d2


def biased_desc():
    """CCU X_2^- (weight 86/100) with its closure X-bar_2^-, the exact rationals printed in
    Tab. ccux_deg_one_col; iteration node k^c_- = k*_- - 1 (Sec. "Domain decomposition:
    iteration of closures")."""
    from fractions import Fraction as Fr
    rhs = ["-43/56000", "1523/126000", "-857/6000", "-39697/36000", "245/288", "2723/6000", "-1459/18000",
           "2899/252000", "-43/56000"]
    clo = ["194871521/170360232000", "-242883881/17036023200", "3813668231/42590058000",
           "-8537761009/18252882000", "-3401756057/4056196000", "40137795113/36505764000",
           "507715327/3650576400", "-338742841/42590058000", "-458269213/511080696000", "16295059/63885087000"]
    return {"order": 6, "a": float(Fr(407, 600)), "lo": -4, "rhs": [float(Fr(v)) for v in rhs],
            "c_sup": float(Fr(407, 600)), "c_lo": -4, "closure": [float(Fr(v)) for v in clo], "kc": 1}


def shift_torch(X, Y, Z):
    """Shift components (beta^x, beta^y, beta^z), both signs inside every block."""
    import torch
    return (torch.cos(X + 2 * Z) + 0.1, torch.sin(Y - X), 0.5 * torch.cos(3 * Y) * torch.sin(Z))


def advect_flops_per_point_axis(n_taps=9, n_iter=1, N=32, g=4):
    """Algorithmic FP64 flops per point, field and axis of the upwinded term: the upwind side's
    FMA chain over the interior taps (2 n_taps), the 1/dx scale, the recurrence FMA and the
    product with beta; plus, per non-final pass of the iteration, the two halo values of a pencil
    (one dense operator row of N + 2g FMAs per side) shared by its N points."""
    return 2 * n_taps + 1 + 2 + 1 + n_iter * 2 * 2 * (N + 2 * g) / N


# ------------------------------------------------------------------ clocks


class ClockSampler:
    """nvidia-smi clock and throttle-reason sampling during the timed region."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.path = None

    def start(self):
        try:
            fd, self.path = tempfile.mkstemp(suffix=".csv")
            os.close(fd)
            self.fh = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.Q}",
                                          "--format=csv,noheader,nounits", "-lms", "100"],
                                         stdout=self.fh, stderr=subprocess.DEVNULL)
        except (OSError, FileNotFoundError):
            self.proc = None

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        self.fh.close()
        sm, mx, reasons = [], None, set()
        names = ("hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap")
        with open(self.path) as fh:
            for line in fh:
                p = [v.strip() for v in line.split(",")]
                if len(p) < 9:
                    continue
                try:
                    sm.append(float(p[1]))
                    mx = float(p[2])
                except ValueError:
                    continue
                for name, v in zip(names, p[5:9]):
                    if v.lower().startswith("active"):
                        reasons.add(name)
        os.unlink(self.path)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": mx, "reasons": sorted(reasons),
                "samples": len(sm)}


# ------------------------------------------------------------------ workloads


def build_workload(name, dev, torch):
    from paper_2302_14858_gb300 import workloads as W
    spec = WORKLOADS[name]
    funcs = W.workload_fields(spec["fields"])[: spec["nf"]]
    tdt = torch.float64 if spec["dtype"] == "f64" else torch.float32
    if spec["kind"] in ("uniform", "advect") and spec.get("mesh") != "boxinbox":
        NM, N, g = spec["NM"], spec["N"], 4
        mesh = W.uniform_mesh(NM, N, g)
        nb, E = NM // N, N + 2 * g
        x = (torch.arange(NM, dtype=torch.float64, device=dev) + 0.5) * (2 * math.pi / NM)
        Z, Y, X = torch.meshgrid(x, x, x, indexing="ij")
        idx = (torch.arange(nb, device=dev)[:, None] * N + torch.arange(-g, N + g, device=dev)[None, :]) % NM
        fields = torch.empty((mesh.nblocks, len(funcs), E, E, E), dtype=tdt, device=dev)
        for q, f in enumerate(funcs):
            fg = _eval_torch(f, X, Y, Z, torch)
            ext = fg[idx[:, None, None, :, None, None], idx[None, :, None, None, :, None],
                     idx[None, None, :, None, None, :]]
            fields[:, q] = ext.reshape(mesh.nblocks, E, E, E).to(tdt)
            del fg, ext
        del X, Y, Z
        return spec, mesh, fields.reshape(-1)
    mesh = W.box_in_box_mesh(4)
    parts = []
    for b in range(mesh.nblocks):
        xs = [torch.as_tensor(c, device=dev, dtype=torch.float64) for c in mesh.coords(b)]
        Z, Y, X = torch.meshgrid(xs[2], xs[1], xs[0], indexing="ij")
        parts.append(torch.stack([_eval_torch(f, X, Y, Z, torch).to(tdt) for f in funcs]).reshape(-1))
    return spec, mesh, torch.cat(parts)


def _eval_torch(f, X, Y, Z, torch):
    from paper_2302_14858_gb300 import workloads as W
    if isinstance(f, W.SineSum):
        out = torch.zeros_like(X)
        for (kx, ky, kz), A, p in zip(f.k, f.A, f.phi):
            out += float(A) * torch.sin(float(kx) * X + float(ky) * Y + float(kz) * Z + float(p))
        return out
    if isinstance(f, W.PeriodicGaussian):
        out = torch.zeros_like(X)
        for sz in (-1, 0, 1):
            for sy in (-1, 0, 1):
                for sx in (-1, 0, 1):
                    r2 = ((X - f.c[0] - sx * W.TWO_PI) ** 2 + (Y - f.c[1] - sy * W.TWO_PI) ** 2
                          + (Z - f.c[2] - sz * W.TWO_PI) ** 2)
                    out += torch.exp(-r2 / (2.0 * f.sigma ** 2))
        return out
    if isinstance(f, W.InverseDistance):
        out = torch.zeros_like(X)
        for c in f.centers:
            d2 = torch.zeros_like(X)
            for v, cc in zip((X, Y, Z), c):
                dv = torch.remainder(torch.abs(v - float(cc)), W.TWO_PI)
                dv = torch.minimum(dv, W.TWO_PI - dv)
                d2 += dv * dv
            out += 1.0 / (torch.sqrt(d2) + 0.5)
        return out
    if isinstance(f, W.Sum):
        out = torch.zeros_like(X)
        for p in f.parts:
            out += _eval_torch(p, X, Y, Z, torch)
        return out
    raise TypeError(type(f))


# ------------------------------------------------------------------ algorithmic work


def banded_flops_per_step(mesh, nf, mask_ops, n_iter, M=3, h=4, g=4, orders=2):
    """FP64 flops of the banded path (RHS FMA chains + Thomas sweeps) for one apply; a mixed
    derivative is solved in ``orders`` orders (2: both, averaged; 1: one order)."""
    def closed(N, pencils):
        rows_int, rows_clo = N - 2, 2
        rhs = rows_int * (2 * (2 * M + 1) - 1) + rows_clo * (2 * (2 * h + 1) - 1)
        return pencils * (rhs + N + 1 + 3 * (N - 1) + 2 * (N - 1))

    def iterated(N, pencils):
        rows = N + 2
        return pencils * (rows * (2 * (2 * M + 1) - 1) + rows + 3 * (N + 3) + 2 * (N + 1))

    def stage(N, pencils):
        return closed(N, pencils) + n_iter * iterated(N, pencils)

    total = 0
    for b in range(mesh.nblocks):
        N = int(mesh.n[b])
        E = N + 2 * g
        for op in mask_ops:
            if len(op) == 2 or op[1] == op[2]:
                total += stage(N, N * N)
            else:
                total += orders * (stage(N, E * N) + stage(N, N * N)) + (2 * N ** 3 if orders == 2 else 0)
    return total * nf


# ------------------------------------------------------------------ CPU baseline (oracle) on every host core

_ORACLE = {}


def _oracle_init(names):
    """Pool worker set-up: one BLAS thread per process, the FP64 scheme coefficients."""
    for v in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS", "NUMEXPR_NUM_THREADS"):
        os.environ[v] = "1"
    from oracle import cfd as C
    with open(os.path.join(ROOT, "tests", "golden", "schemes.json")) as fh:
        S = json.load(fh)
    for slot, name in zip(("s1", "s2"), names):
        e = S[name]
        _ORACLE[slot] = C.Sch(e["d"], e["a"], tuple(e["rhs"]), tuple(e["closure"]))


def _oracle_task(task):
    """One unit of oracle work on one field, timed inside the worker (data generation excluded):
    closed blocks of the workload's mesh, each applied on its own (apply_block), or, with the
    hybrid iteration, a periodic sub-problem of 2 x 2 x 2 blocks (apply_uniform).  Returns
    (point-ops, seconds)."""
    from oracle import cfd as C
    from paper_2302_14858_gb300 import workloads as W
    f = W.workload_fields(task["fields"])[task["field"]]
    ops, g = task["ops"], 4
    s1, s2 = _ORACLE["s1"], _ORACLE["s2"]
    if task["mesh"] == "uniform" and task["NM"] == task["N"]:
        # one periodic block: the undecomposed cyclic scheme along each requested axis
        NM = task["NM"]
        dx = 2 * np.pi / NM
        x = (np.arange(NM) + 0.5) * dx
        Z, Y, X = np.meshgrid(x, x, x, indexing="ij")
        fg = f(X, Y, Z)
        t0 = time.perf_counter()
        for _ in range(task["reps"]):
            for op in ops:
                ax = {"x": 2, "y": 1, "z": 0}[op[1]]
                C.global_periodic(np.moveaxis(fg, ax, 0), s1 if len(op) == 2 else s2, dx)
        return NM ** 3 * len(ops) * task["reps"], time.perf_counter() - t0
    if task["n_iter"] == 0:
        mesh = W.box_in_box_mesh(g) if task["mesh"] == "boxinbox" else W.uniform_mesh(task["NM"], task["N"], g)
        data = W.sample(mesh, [f], blocks=task["blocks"])
        t0 = time.perf_counter()
        units = 0
        for _ in range(task["reps"]):
            for b, arr in zip(task["blocks"], data):
                N = int(mesh.n[b])
                C.apply_block(arr[0], s1, s2, mesh.dx[b], N, g, ops)
                units += N ** 3 * len(ops)
        return units, time.perf_counter() - t0
    N = task["N"]
    NS = 2 * N
    dx = 2 * np.pi / task["NM"]
    x = (np.arange(NS) + 0.5) * dx
    Z, Y, X = np.meshgrid(x, x, x, indexing="ij")
    ext = C.ghost_fill_3d(f(X, Y, Z), N, g)
    t0 = time.perf_counter()
    for _ in range(task["reps"]):
        C.apply_uniform(ext, s1, s2, (dx, dx, dx), N, g, ops, task["n_iter"])
    return NS ** 3 * len(ops) * task["reps"], time.perf_counter() - t0


class OraclePool:
    """The oracle (numpy FP64, as it stands) on all host cores: a spawn-started process pool (no
    process is forked from one that has used the GPU) running independent tasks of the same
    workload: same block size, fields, ops and iteration count."""

    def __init__(self, spec):
        import multiprocessing as mp
        self.spec = spec
        self.procs = len(os.sched_getaffinity(0)) if hasattr(os, "sched_getaffinity") else (os.cpu_count() or 1)
        names = ("P2_d1", "P2_d2") if spec.get("scheme") == "P12" else ("Q13_1_d1", "Q13_1_d2")
        _oracle_init(names)                       # the in-process calibration uses the same set-up
        self.pool = mp.get_context("spawn").Pool(self.procs, initializer=_oracle_init, initargs=(names,))
        self.rng = np.random.default_rng(2302)

    def _tasks(self, n, reps=1):
        sp = self.spec
        from paper_2302_14858_gb300 import workloads as W
        box = sp["kind"] != "uniform"
        mesh = W.box_in_box_mesh(4) if box else None
        nb = mesh.nblocks if box else (sp["NM"] // sp["N"]) ** 3
        ops = ("dx",) if sp.get("ops") == "dx" else OPS9
        per = 1 if box else max(1, min(8, nb))
        out = []
        for k in range(n):
            out.append({"kind": sp["kind"], "mesh": "boxinbox" if box else "uniform", "NM": sp.get("NM", 128),
                        "N": sp.get("N", 16), "fields": sp["fields"], "field": k % sp["nf"], "ops": ops,
                        "n_iter": sp["n_iter"], "reps": reps,
                        "blocks": [int(b) for b in self.rng.choice(nb, size=per, replace=False)]})
        return out

    def run(self, seconds):
        one = _oracle_task(self._tasks(1)[0])[1]          # calibration, in this process
        reps = max(1, int(0.05 / max(one, 1e-6)))         # tasks of ~50 ms at least
        n = max(self.procs, int(math.ceil(seconds / (one * reps))) * self.procs)
        tasks = self._tasks(n, reps)
        t0 = time.perf_counter()
        res = self.pool.map(_oracle_task, tasks, chunksize=1)
        wall = time.perf_counter() - t0
        units = sum(r[0] for r in res)
        busy = sum(r[1] for r in res)
        t = tasks[0]
        each = (f"the periodic {t['NM']}^3 block, cyclic scheme" if t["mesh"] == "uniform" and t["NM"] == t["N"]
                else f"{len(t['blocks'])} closed block(s) of the workload's mesh" if t["n_iter"] == 0
                else f"a periodic {2 * t['N']}^3 sub-problem of 2x2x2 blocks, n_iter={t['n_iter']}")
        what = f"{len(tasks)} tasks on {self.procs} processes; each: {each}, 1 field, {len(t['ops'])} op(s)"
        return {"value": units / wall / 1e9, "unit": "Gpoint-ops/s", "cores": self.procs, "kind": "oracle",
                "sample": what, "same_config": True, "host_cores": os.cpu_count(),
                "per_core_value": units / busy / 1e9, "wall_s": round(wall, 2)}

    def close(self):
        self.pool.terminate()
        self.pool.join()


OPS9 = ("dx", "dy", "dz", "dxx", "dyy", "dzz", "dxy", "dxz", "dyz")


def cpu_baseline(spec, seconds=12.0):
    """Time the oracle on a bounded sample of the workload (host cores).  The derivative
    workloads run on every core (OraclePool); the time-stepping workloads, whose blocks are
    coupled every stage, on one process."""
    if spec["kind"] in ("uniform", "boxinbox"):
        pool = OraclePool(spec)
        try:
            return pool.run(seconds)
        finally:
            pool.close()
    for v in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS"):
        os.environ.setdefault(v, "1")
    from oracle import cfd as C
    from paper_2302_14858_gb300 import workloads as W
    with open(os.path.join(ROOT, "tests", "golden", "schemes.json")) as fh:
        S = json.load(fh)
    e1, e2 = S["Q13_1_d1"], S["Q13_1_d2"]
    s1 = C.Sch(1, e1["a"], tuple(e1["rhs"]), tuple(e1["closure"]))
    s2 = C.Sch(2, e2["a"], tuple(e2["rhs"]), tuple(e2["closure"]))
    g = 4
    if spec["kind"] == "wave" and spec.get("shift") is not None:
        from oracle import biased as BO
        from oracle import timestep as TS
        d = biased_desc()
        bs = BO.Biased(d["a"], d["lo"], tuple(d["rhs"]), d["c_sup"], d["c_lo"], tuple(d["closure"]), d["kc"])
        NS, N = 64, spec["N"]
        pw = W.plane_waves(2302 + 5, spec["modes"], spec["kmax"])
        dx = 2 * np.pi / NS
        x = (np.arange(NS) + 0.5) * dx
        Z, Y, X = np.meshgrid(x, x, x, indexing="ij")
        p, k = pw.phi_at(0.0, X, Y, Z), pw.K_at(0.0, X, Y, Z)
        beta = [np.full_like(X, v) for v in spec["shift"]]
        coef = TS.lsrk2s_rk4_float()
        units, reps = 0, 0
        t0 = time.perf_counter()
        while True:
            p, k = TS.shifted_wave_lsrk_step(p, k, beta, 0.25 * dx, coef, s2, bs, (dx, dx, dx), N, g,
                                             spec["n_iter"], 0.04, 4)
            units += 5 * NS ** 3 * 4
            reps += 1
            if time.perf_counter() - t0 > seconds:
                break
        el = time.perf_counter() - t0
        return {"value": units / el / 1e9, "unit": "Gpoint-ops/s", "cores": 1, "kind": "oracle",
                "sample": f"oracle shifted_wave_lsrk_step, {NS}^3 as {(NS // N) ** 3} blocks of {N}^3, {reps} steps"}
    if spec["kind"] == "wave":
        # sample: one RK4 step of the oracle on 64^3 as 8 blocks of 32^3 (units: 3 ops x points x 4 stages)
        NS, N = 64, spec["N"]
        pw = W.plane_waves(2302 + 5, spec["modes"], spec["kmax"])
        dx = 2 * np.pi / NS
        x = (np.arange(NS) + 0.5) * dx
        Z, Y, X = np.meshgrid(x, x, x, indexing="ij")
        p, k = pw.phi_at(0.0, X, Y, Z), pw.K_at(0.0, X, Y, Z)
        units, reps = 0, 0
        t0 = time.perf_counter()
        while True:
            p, k = C.wave_rk4_step(p, k, 0.25 * dx, s2, (dx, dx, dx), N, g, spec["n_iter"])
            units += 3 * NS ** 3 * 4
            reps += 1
            if time.perf_counter() - t0 > seconds:
                break
        el = time.perf_counter() - t0
        return {"value": units / el / 1e9, "unit": "Gpoint-ops/s", "cores": 1, "kind": "oracle",
                "sample": f"oracle wave_rk4_step, {NS}^3 as {(NS // N) ** 3} blocks of {N}^3, {reps} RK4 steps"}
    if spec["kind"] == "adv2d":
        from oracle import biased as BO
        from oracle import timestep as TS
        d = biased_desc()
        bs = BO.Biased(d["a"], d["lo"], tuple(d["rhs"]), d["c_sup"], d["c_lo"], tuple(d["closure"]), d["kc"])
        NS, N = 64, spec["N"]
        dx = 2 * np.pi / spec["NM"]
        x = (np.arange(NS) + 0.5) * dx
        z = (np.arange(N) + 0.5) * dx
        Z, Y, X = np.meshgrid(z, x, x, indexing="ij")
        u = adv2d_profile(X, Y)
        phi = math.radians(spec["angle_deg"])
        beta = [np.full_like(X, -math.cos(phi)), np.full_like(X, -math.sin(phi)), 0 * X]
        coef = TS.lsrk2s_rk4_float()
        units, reps = 0, 0
        t0 = time.perf_counter()
        while True:
            u = TS.advect_lsrk_step(u, beta, spec["cfl"] * dx, coef, bs, (dx, dx, dx), N, g, spec["n_iter"], 0.04, 4)
            units += NS * NS * N * 4
            reps += 1
            if time.perf_counter() - t0 > seconds:
                break
        el = time.perf_counter() - t0
        return {"value": units / el / 1e9, "unit": "Gpoint-ops/s", "cores": 1, "kind": "oracle",
                "sample": f"oracle advect_lsrk_step, {NS}x{NS}x{N} as {(NS // N) ** 2} blocks of {N}^3, {reps} steps"}
    if spec["kind"] == "advect":
        from oracle import biased as BO
        d = biased_desc()
        bs = BO.Biased(d["a"], d["lo"], tuple(d["rhs"]), d["c_sup"], d["c_lo"], tuple(d["closure"]), d["kc"])
        NS, N = 64, spec["N"]
        f = W.workload_fields(spec["fields"])[0]
        dx = 2 * np.pi / NS
        x = (np.arange(NS) + 0.5) * dx
        Z, Y, X = np.meshgrid(x, x, x, indexing="ij")
        ext = C.ghost_fill_3d(f(X, Y, Z), N, g)
        beta = [C.global_to_blocks(v, N) for v in (np.cos(X + 2 * Z) + 0.1, np.sin(Y - X),
                                                   0.5 * np.cos(3 * Y) * np.sin(Z))]
        units, reps = 0, 0
        t0 = time.perf_counter()
        while True:
            BO.advect_uniform(ext, beta, bs, (dx, dx, dx), N, g, spec["n_iter"])
            units += NS ** 3
            reps += 1
            if time.perf_counter() - t0 > seconds:
                break
        el = time.perf_counter() - t0
        return {"value": units / el / 1e9, "unit": "Gpoint-ops/s", "cores": 1, "kind": "oracle",
                "sample": f"oracle advect_uniform, 1 field, {NS}^3 as {(NS // N) ** 3} blocks of {N}^3, "
                          f"n_iter={spec['n_iter']}, {reps} reps"}
    raise ValueError(spec["kind"])


# ------------------------------------------------------------------ main


def blocks_iter_ok(mesh) -> bool:
    """Every block has same-size face neighbours along every axis (the hybrid iteration's need)."""
    faces = [i for i, d in enumerate(__import__("paper_2302_14858_gb300.workloads", fromlist=["DIRS"]).DIRS)
             if sum(abs(v) for v in d) == 1]
    return bool(np.all(mesh.neighbors[:, faces] >= 0))


def algorithmic_bytes(nint, nf, nops, elem):
    """Minimal HBM traffic of one apply: read every field value once, write every output once."""
    return nint * nf * elem * (1 + nops)


def tc_flops(mesh, nf, slices_pairs, g=4):
    """Tensor-core flops of the dense path per apply (9 ops, closures only, one mixed order)."""
    total = 0
    for b in range(mesh.nblocks):
        N = int(mesh.n[b])
        E = N + 2 * g
        Kp = (E + 15) // 16 * 16
        pen = N * N
        total += 3 * pen * 2 * N * Kp * 2 * slices_pairs            # d_a and d_aa tiles
        total += 3 * (E * N * N * Kp * 2 + pen * N * Kp * 2) * slices_pairs  # mixed: two stages
    return total * nf


def max_abs_diff_per_field_op(out, ref, mesh, nf, nops, torch):
    """max |out - ref| and max |ref| per (field, op) over all blocks (outputs [block][field][op][N^3])."""
    errs = torch.zeros(nf, nops, dtype=torch.float64, device=out.device)
    maxs = torch.zeros_like(errs)
    off, b = 0, 0
    while b < mesh.nblocks:
        e = b
        while e < mesh.nblocks and mesh.n[e] == mesh.n[b]:
            e += 1
        n3 = int(mesh.n[b]) ** 3
        cnt = (e - b) * nf * nops * n3
        o = out[off:off + cnt].view(e - b, nf, nops, n3)
        r = ref[off:off + cnt].view(e - b, nf, nops, n3)
        for q in range(nf):   # per field keeps the temporaries small
            errs[q] = torch.maximum(errs[q], (o[:, q].double() - r[:, q].double()).abs().amax(dim=(0, 2)))
            maxs[q] = torch.maximum(maxs[q], r[:, q].double().abs().amax(dim=(0, 2)))
        off += cnt
        b = e
    return errs, maxs


def max_over_ranks(ms: float, device=None) -> float:
    """The job's time is the slowest rank's: all-reduce MAX over the process group (identity on
    a single process).  ``device`` is the CUDA device for NCCL, None for a CPU (gloo) group."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return ms
    t = torch.tensor([ms], dtype=torch.float64, device=device if device is not None else "cpu")
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def whole_job_value(units_per_rank: float, world: int, ms: float) -> float:
    """Whole-job throughput in G units/s: every rank processes units_per_rank in ms (the max)."""
    return units_per_rank * world / (ms * 1e-3) / 1e9


def e2e_pipelined(torch, dev, host_in, dev_in, host_out, dev_out, compute, steps, chunks=4):
    """End-to-end steps with two in flight: the host->device copy of step k+1 and the
    device->host copy of step k-1 overlap the compute of step k (streams ordered by events,
    device buffers and host results double-buffered).  Each copy is split into ``chunks`` parts
    on their own streams so that several copy engines work on it.  Returns ms per step from
    the first copy in to the last copy out."""
    s_c = torch.cuda.Stream(dev)
    s_in = [torch.cuda.Stream(dev) for _ in range(chunks)]
    s_out = [torch.cuda.Stream(dev) for _ in range(chunks)]
    ev = lambda: [[torch.cuda.Event() for _ in range(chunks)] for _ in range(2)]
    h2d, d2h = ev(), ev()
    comp = [torch.cuda.Event(), torch.cuda.Event()]

    def parts(n):
        b = [n * c // chunks for c in range(chunks + 1)]
        return list(zip(b[:-1], b[1:]))

    pin, pout = parts(host_in.numel()), parts(host_out[0].numel())
    start, end = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    start.record(s_in[0])
    for s in s_in[1:] + s_out:
        s.wait_event(start)
    for k in range(steps):
        i = k & 1
        for c, (a, b) in enumerate(pin):
            if k >= 2:
                s_in[c].wait_event(comp[i])   # the compute that read dev_in[i] is done
            with torch.cuda.stream(s_in[c]):
                dev_in[i][a:b].copy_(host_in[a:b], non_blocking=True)
            h2d[i][c].record(s_in[c])
            s_c.wait_event(h2d[i][c])
        if k >= 2:
            for c in range(chunks):
                s_c.wait_event(d2h[i][c])     # dev_out[i] has been copied out
        compute(dev_in[i], dev_out[i], s_c)
        comp[i].record(s_c)
        for c, (a, b) in enumerate(pout):
            s_out[c].wait_event(comp[i])
            with torch.cuda.stream(s_out[c]):
                host_out[i][a:b].copy_(dev_out[i][a:b], non_blocking=True)
            d2h[i][c].record(s_out[c])
    for s in s_out[1:]:
        e = torch.cuda.Event()
        e.record(s)
        s_out[0].wait_event(e)
    end.record(s_out[0])
    torch.cuda.synchronize()
    return start.elapsed_time(end) / steps


def timed(step, steps, stream, torch):
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(steps):
        step()
    e1.record(stream)
    torch.cuda.synchronize()
    return e0.elapsed_time(e1) / steps


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=200)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--workload", default=DEFAULT_WORKLOAD, choices=sorted(WORKLOADS))
    ap.add_argument("--prec", default="tc_bf16_exact", choices=sorted(PREC))
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--n-iter", type=int, default=None)
    ap.add_argument("--compare-steps", type=int, default=5, help="timed steps of the FP64 banded comparison")
    ap.add_argument("--no-compare", action="store_true")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-autotune", action="store_true", help="tensor-core path: default launch choices")
    ap.add_argument("--graph", action="store_true", help="also time the step replayed from a captured CUDA graph")
    ap.add_argument("--integrator", default="erk4", choices=["erk4", "lsrk2s"],
                    help="wave workload: classical RK4, or the 2S low-storage RK with Kreiss-Oliger dissipation")
    ap.add_argument("--sigma", type=float, default=0.04, help="Kreiss-Oliger strength for --integrator lsrk2s")
    ap.add_argument("--ko-r", type=int, default=4, help="Kreiss-Oliger order 2r for --integrator lsrk2s")
    args = ap.parse_args()

    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    spec = dict(WORKLOADS[args.workload])
    if args.n_iter is not None:
        spec["n_iter"] = args.n_iter

    if args.impl == "reference":
        return run_reference(args, spec, rank)
    if spec["kind"] == "wave":
        return run_wave(args, spec)
    if spec["kind"] == "advect":
        return run_advect(args, spec)
    if spec["kind"] == "adv2d":
        return run_adv2d(args, spec)

    import torch
    if world > 1:
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl")
    dev = torch.device("cuda", local)
    torch.cuda.set_device(dev)

    from paper_2302_14858_gb300 import cfd
    d1, d2 = scheme_descs(spec.get("scheme", "Q13"))
    scheme = cfd.cfd_scheme_create(d1, d2)
    spec_, mesh, fields = build_workload(args.workload, dev, torch)
    dtype = cfd.CFD_F64 if spec["dtype"] == "f64" else cfd.CFD_F32
    blocks = cfd.cfd_blocks_bind(scheme, mesh.n, mesh.dx, mesh.neighbors, mesh.g, dtype)
    nf = spec["nf"]
    op_names = ("dx",) if spec.get("ops") == "dx" else tuple(cfd.OPS)
    mask = cfd.op_mask(list(op_names))
    nops = len(op_names)
    prec = PREC[args.prec]
    n_iter = spec["n_iter"]
    nint = int(sum(int(n) ** 3 for n in mesh.n))
    units = nint * nf * nops
    out = torch.empty(units, dtype=fields.dtype, device=dev)
    ws = max(cfd.cfd_apply_workspace(blocks, nf, mask, prec, n_iter),
             cfd.cfd_apply_workspace(blocks, nf, mask, cfd.CFD_FP64_BANDED, n_iter))
    work = torch.empty(max(ws, 256), dtype=torch.uint8, device=dev)
    stream = torch.cuda.current_stream(dev)

    def step():
        cfd.cfd_exchange_ghosts(blocks, fields, nf, stream)
        cfd.cfd_apply(blocks, fields, nf, mask, prec, n_iter, out, work, stream)

    # the autotuner picks each kernel's staging and tile order on these inputs (untimed)
    autotune = None
    if prec != PREC["fp64_banded"] and not args.no_autotune:
        cfd.cfd_exchange_ghosts(blocks, fields, nf, stream)
        cfd.cfd_autotune(blocks, fields, nf, mask, prec, n_iter, out, work, stream)
        autotune = cfd.cfd_autotune_report(blocks)
    for _ in range(args.warmup):
        step()
    cfd.cfd_sync_status(blocks, stream)
    torch.cuda.synchronize()

    def barrier():
        if world > 1:
            import torch.distributed as dist
            dist.barrier()

    clocks = ClockSampler(local)
    launches0 = cfd.cfd_kernel_launches()
    barrier()
    torch.cuda.synchronize()
    clocks.start()
    time.sleep(0.3)
    ms_step = timed(step, args.steps, stream, torch)
    barrier()
    clk = clocks.stop()
    cfd.cfd_sync_status(blocks, stream)
    launches = cfd.cfd_kernel_launches() - launches0
    # per-launch CUDA events around every kernel, in a second timed region of the same step
    # (kept out of the headline region: the event records sit between the launches)
    prof_steps = max(3, min(args.steps, 50))
    cfd.cfd_profile_enable(True)
    torch.cuda.synchronize()
    ms_prof = timed(step, prof_steps, stream, torch)
    prof = {name: cfd.cfd_profile_read(fid) for name, fid in cfd.KERNEL_FAMILIES.items()}
    cfd.cfd_profile_enable(False)
    ms_step = max_over_ranks(ms_step, dev)
    value = whole_job_value(units, world, ms_step)
    ms_total = ms_prof * prof_steps

    # roofline of the dominant kernel family, from the per-launch event times of the timed region
    fam, (nl, tl) = max(prof.items(), key=lambda kv: kv[1][1])
    elem = fields.element_size()
    if fam == "line":
        fl = banded_flops_per_step(mesh, nf, op_names, n_iter) * prof_steps
        achieved = fl / (tl * 1e-3) / 1e9
        roof = {"kernel": "k_line (FP64 banded pencil solve)", "bound": "alu", "achieved": round(achieved, 2),
                "peak": FP64_NOMINAL_GFLOPS, "unit": "GFLOP/s", "frac": round(achieved / FP64_NOMINAL_GFLOPS, 4),
                "peak_source": "FP64 nominal 1.25 TFLOP/s (profiling recipe table; 1.256 measured)",
                "traffic": None}
    else:
        peaks = {}
        try:
            with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as fh:
                peaks = json.load(fh)
        except OSError:
            pass
        hbm = float(peaks.get("hbm_gbs", 6800.0))
        byts = algorithmic_bytes(nint, nf, nops, elem) * prof_steps
        achieved = byts / (tl * 1e-3) / 1e9
        pairs = 15 if prec == PREC["tc_bf16_exact"] else 3
        tcf = tc_flops(mesh, nf, pairs) * prof_steps / (tl * 1e-3) / 1e12 if nops == 9 else None
        roof = {"kernel": "k_dense (tcgen05 BF16 digit-slice GEMM)", "bound": "hbm", "achieved": round(achieved, 1),
                "peak": hbm, "unit": "GB/s", "frac": round(achieved / hbm, 4),
                "peak_source": "measured" if "hbm_gbs" in peaks else "fallback",
                "algorithmic_bytes_per_point_op": round(elem * (1 + nops) / nops, 3),
                "tensor_tflops": round(tcf, 1) if tcf else None,
                "tensor_frac_of_bf16_peak": round(tcf / float(peaks.get("bf16_tflops", 1900.0)), 4) if tcf else None,
                "traffic": MEASURED_TRAFFIC.get((args.workload, args.prec, n_iter)),
                "algorithmic_bytes_per_launch": round(algorithmic_bytes(nint, nf, nops, elem) / max(nl / prof_steps, 1))}
    if roof.get("traffic") and roof.get("unit") == "GB/s":
        # the DRAM bytes the kernel actually moves per launch, over the same event time
        dram = roof["traffic"] / (tl / max(nl, 1) * 1e-3) / 1e9
        roof.update({"traffic_gbs": round(dram, 1), "traffic_frac": round(dram / roof["peak"], 4),
                     "traffic_over_algorithmic": round(roof["traffic"] / roof["algorithmic_bytes_per_launch"], 3)})
    roof.update({"launches_per_step": nl / prof_steps, "avg_launch_ms": round(tl / max(nl, 1), 5),
                 "share_of_step": round(tl / ms_total, 4), "events_region": {"steps": prof_steps,
                                                                          "ms_per_step": round(ms_prof, 5)}})

    # The FP64 banded solve on the same inputs: speed and max relative difference per (field, op).
    # Two forms: the paper's symmetrised mixed derivatives (both orders, averaged) and one order,
    # the work the tensor-core path does (cfd_blocks_set_mixed_order; equal on these meshes to
    # rounding).  The speed-up is quoted against the one-order form (equal work).
    compare = None
    if not args.no_compare and prec != PREC["fp64_banded"]:
        ref = torch.empty_like(out)

        def step64():
            cfd.cfd_exchange_ghosts(blocks, fields, nf, stream)
            cfd.cfd_apply(blocks, fields, nf, mask, cfd.CFD_FP64_BANDED, n_iter, ref, work, stream)

        def line_roofline(orders):
            # k_line alone, per-launch CUDA events over a few more steps (FP64-pipe bound)
            cfd.cfd_profile_enable(True)
            torch.cuda.synchronize()
            ms = timed(step64, args.compare_steps, stream, torch)
            nl, tl = cfd.cfd_profile_read(cfd.KERNEL_FAMILIES["line"])
            cfd.cfd_profile_enable(False)
            fl = banded_flops_per_step(mesh, nf, op_names, n_iter, orders=orders) * args.compare_steps
            ach = fl / (tl * 1e-3) / 1e9
            return {"kernel": "k_line (FP64 banded pencil solve)", "bound": "alu", "achieved": round(ach, 1),
                    "peak": FP64_NOMINAL_GFLOPS, "unit": "GFLOP/s", "frac": round(ach / FP64_NOMINAL_GFLOPS, 4),
                    "launches_per_step": nl / args.compare_steps, "avg_launch_ms": round(tl / max(nl, 1), 5),
                    "share_of_step": round(tl / (ms * args.compare_steps), 4)}

        step64()
        torch.cuda.synchronize()
        ms64 = timed(step64, args.compare_steps, stream, torch)
        roof64 = line_roofline(2)
        one_order = blocks.handle is not None and nops == 9
        ms64_one = roof64_one = None
        if one_order:
            try:
                cfd.cfd_blocks_set_mixed_order(blocks, True)
                step64()
                torch.cuda.synchronize()
                ms64_one = timed(step64, args.compare_steps, stream, torch)
                roof64_one = line_roofline(1)
            except cfd.CfdError:
                ms64_one = None
            cfd.cfd_blocks_set_mixed_order(blocks, False)
            step64()
        step()
        torch.cuda.synchronize()
        errs, maxs = max_abs_diff_per_field_op(out, ref, mesh, nf, nops, torch)
        rel = (errs / maxs).cpu().numpy()
        worst = float(rel.max())
        base_ms = ms64_one if ms64_one else ms64
        compare = {"fp64_banded": {"value": round(units / (ms64 * 1e-3) / 1e9, 4), "ms_per_step": round(ms64, 4),
                                   "mixed": "symmetrised (both orders averaged)", "roofline": roof64},
                   "fp64_banded_one_order": ({"value": round(units / (ms64_one * 1e-3) / 1e9, 4),
                                              "ms_per_step": round(ms64_one, 4), "mixed": "one order",
                                              "roofline": roof64_one}
                                             if ms64_one else None),
                   "speedup_vs_fp64_banded": round(base_ms / ms_step, 3),
                   "speedup_basis": "one-order FP64 banded (equal work)" if ms64_one else "FP64 banded",
                   "speedup_vs_fp64_banded_symmetrised": round(ms64 / ms_step, 3),
                   "max_rel_err_vs_fp64_banded": worst,
                   "max_rel_err_per_op": {op: float(rel[:, i].max()) for i, op in enumerate(op_names)}}
        del ref

    # the paper's working setting, one hybrid iteration (Sec. "Domain decomposition: iteration of
    # closures"), on the same workload when the headline runs closures only
    iter1 = None
    if n_iter == 0 and mesh.nblocks > 1 and blocks_iter_ok(mesh):
        ws1 = cfd.cfd_apply_workspace(blocks, nf, mask, prec, 1)
        work1 = torch.empty(max(ws1, 256), dtype=torch.uint8, device=dev) if ws1 > work.numel() else work

        def step1():
            cfd.cfd_exchange_ghosts(blocks, fields, nf, stream)
            cfd.cfd_apply(blocks, fields, nf, mask, prec, 1, out, work1, stream)

        for _ in range(max(2, args.warmup)):
            step1()
        torch.cuda.synchronize()
        n1 = max(3, min(args.steps, 30))
        cfd.cfd_profile_enable(True)
        ms1 = timed(step1, n1, stream, torch)
        nl1, tl1 = cfd.cfd_profile_read(cfd.KERNEL_FAMILIES["dense"]) if prec != PREC["fp64_banded"] else \
            cfd.cfd_profile_read(cfd.KERNEL_FAMILIES["line"])
        nh1, th1 = cfd.cfd_profile_read(cfd.KERNEL_FAMILIES["dense_halo"])
        cfd.cfd_profile_enable(False)
        cfd.cfd_sync_status(blocks, stream)
        iter1 = {"n_iter": 1, "value": round(whole_job_value(units, world, max_over_ranks(ms1, dev)), 4),
                 "ms_per_step": round(ms1, 5), "launches_per_step": round((nl1 + nh1) / n1, 2)}
        if fam != "line" and tl1 > 0:
            a1 = algorithmic_bytes(nint, nf, nops, elem) * n1 / ((tl1 + th1) * 1e-3) / 1e9
            iter1["roofline"] = {"achieved": round(a1, 1), "unit": "GB/s", "frac": round(a1 / hbm, 4),
                                 "how": "algorithmic bytes per step / time per step of the final passes (k_dense) "
                                        "and the halo passes (k_halo_rows)",
                                 "k_dense_ms_per_step": round(tl1 / n1, 4),
                                 "k_halo_rows": {"launches_per_step": round(nh1 / n1, 2),
                                                 "ms_per_step": round(th1 / n1, 4)}}
        del work1

    # the same step captured once into a CUDA graph and replayed (launch overhead removed)
    graph = None
    if args.graph:
        side = torch.cuda.Stream(dev)
        side.wait_stream(stream)

        def step_cur():
            cur = torch.cuda.current_stream(dev)
            cfd.cfd_exchange_ghosts(blocks, fields, nf, cur)
            cfd.cfd_apply(blocks, fields, nf, mask, prec, n_iter, out, work, cur)

        with torch.cuda.stream(side):
            step_cur()
        stream.wait_stream(side)
        torch.cuda.synchronize()
        g = torch.cuda.CUDAGraph()
        with torch.cuda.graph(g, stream=side):
            step_cur()
        for _ in range(args.warmup):
            g.replay()
        torch.cuda.synchronize()
        ms_g = timed(g.replay, args.steps, torch.cuda.current_stream(dev), torch)
        cfd.cfd_sync_status(blocks, stream)
        graph = {"value": round(units * world / (ms_g * 1e-3) / 1e9, 4), "ms_per_step": round(ms_g, 5),
                 "launches_per_step": round(launches / args.steps, 2)}

    # end-to-end through the C ABI with host buffers
    e2e = None
    if not args.no_e2e:
        host_in = torch.empty(fields.numel(), dtype=fields.dtype, pin_memory=True)
        host_in.copy_(fields)
        host_out = torch.empty(out.numel(), dtype=out.dtype, pin_memory=True)

        def step_e2e():
            fields.copy_(host_in, non_blocking=True)
            step()
            host_out.copy_(out, non_blocking=True)

        step_e2e()
        torch.cuda.synchronize()
        barrier()
        n_e2e = max(3, min(20, args.steps // 10))
        ms_serial = timed(step_e2e, n_e2e, stream, torch)
        # the same with two steps in flight (copies in and out overlap the compute and each other)
        fields2, out2 = torch.empty_like(fields), torch.empty_like(out)
        host_out2 = torch.empty(out.numel(), dtype=out.dtype, pin_memory=True)

        def compute(fin, fout, st):
            cfd.cfd_exchange_ghosts(blocks, fin, nf, st)
            cfd.cfd_apply(blocks, fin, nf, mask, prec, n_iter, fout, work, st)

        ms_pipe = e2e_pipelined(torch, dev, host_in, [fields, fields2], [host_out, host_out2], [out, out2],
                                compute, n_e2e)
        ms_pipe = max_over_ranks(ms_pipe, dev)
        ms_serial = max_over_ranks(ms_serial, dev)
        # both are ways a caller can drive the API; the host link (about 200 GB/s each way on the
        # GPU machines, shared with other tenants) decides which is faster on a given run
        best = min(ms_pipe, ms_serial)
        e2e = {"value": round(whole_job_value(units, world, best), 4), "unit": "Gpoint-ops/s",
               "h2d_bytes_per_step": host_in.numel() * host_in.element_size(),
               "d2h_bytes_per_step": host_out.numel() * host_out.element_size(),
               "ms_per_step": round(best, 4), "strategy": "pipelined" if ms_pipe <= ms_serial else "serial",
               "pipelined": {"value": round(whole_job_value(units, world, ms_pipe), 4), "ms_per_step": round(ms_pipe, 4),
                             "how": "two steps in flight, copies overlap compute, each copy in 4 concurrent parts"},
               "serial": {"value": round(whole_job_value(units, world, ms_serial), 4),
                          "ms_per_step": round(ms_serial, 4)}}
        del fields2, out2, host_out2

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        cpu = cpu_baseline(spec)

    if rank == 0:
        in_bytes = fields.numel() * fields.element_size()
        if e2e is not None:
            e2e["bound"] = "host link (pinned copies of every step's inputs and outputs)"
        line = {
            "metric": METRIC, "value": round(value, 4), "unit": "Gpoint-ops/s", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(ms_step, 5),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": arithmetic_name(prec, spec["dtype"]), "data": "synthetic (seeded analytic fields)",
            "config": {"workload": args.workload, "path": args.prec, "n_iter": n_iter, "fields": nf, "ops": nops,
                       "blocks": mesh.nblocks, "points_per_field": nint,
                       "l2": "inputs larger than L2" if in_bytes > L2_BYTES else "inputs fit L2",
                       "input_bytes": in_bytes, "parallelism": f"replicas x{world}"},
            "roofline": roof, "compare": compare, "n_iter1": iter1, "cpu_baseline": cpu, "e2e": e2e,
            "graph": graph, "autotune": autotune, "gpu_launches": int(launches), "clocks": clk,
        }
        print(json.dumps(line))
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


def run_advect(args, spec):
    """Upwinded shift advection: Gpoint-ops/s = interior points x fields (one advective term
    sum_i beta^i d_i f each) / step time; a step is the ghost exchange of the fields plus
    cfd_advect (FP64 biased pencil solves, both biases, every axis, with iteration)."""
    import torch
    from paper_2302_14858_gb300 import cfd
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl")
    dev = torch.device("cuda", local)
    torch.cuda.set_device(dev)
    scheme = cfd.cfd_scheme_create(scheme_descs()[0], None)
    cfd.cfd_scheme_set_biased(scheme, biased_desc())
    _, mesh, fields = build_workload(args.workload, dev, torch)
    N, g = spec["N"], 4
    E = N + 2 * g
    box = spec.get("mesh") == "boxinbox"
    tdt = fields.dtype
    if box:
        parts = []
        for b in range(mesh.nblocks):
            xs = [torch.as_tensor(cc, device=dev, dtype=torch.float64) for cc in mesh.coords(b)]
            Zb, Yb, Xb = torch.meshgrid(xs[2], xs[1], xs[0], indexing="ij")
            parts.append(torch.stack(shift_torch(Xb, Yb, Zb)).to(tdt).reshape(-1))
        beta = torch.cat(parts)
    else:
        NM = spec["NM"]
        nb = NM // N
        x = (torch.arange(NM, dtype=torch.float64, device=dev) + 0.5) * (2 * math.pi / NM)
        Z, Y, X = torch.meshgrid(x, x, x, indexing="ij")
        idx = (torch.arange(nb, device=dev)[:, None] * N + torch.arange(-g, N + g, device=dev)[None, :]) % NM
        beta = torch.empty((mesh.nblocks, 3, E, E, E), dtype=tdt, device=dev)
        for i, bg in enumerate(shift_torch(X, Y, Z)):
            beta[:, i] = bg[idx[:, None, None, :, None, None], idx[None, :, None, None, :, None],
                            idx[None, None, :, None, None, :]].reshape(mesh.nblocks, E, E, E).to(tdt)
        del X, Y, Z
        beta = beta.reshape(-1)
    blocks = cfd.cfd_blocks_bind(scheme, mesh.n, mesh.dx, mesh.neighbors, g,
                                 cfd.CFD_F32 if spec["dtype"] == "f32" else cfd.CFD_F64)
    nf, n_iter = spec["nf"], spec["n_iter"]
    nint = int(sum(int(n) ** 3 for n in mesh.n))
    units = nint * nf
    out = torch.empty(units, dtype=tdt, device=dev)
    prec = PREC[args.prec]
    ws = max(cfd.cfd_biased_workspace(blocks, nf, prec, n_iter),
             cfd.cfd_biased_workspace(blocks, nf, cfd.CFD_FP64_BANDED, n_iter))
    work = torch.empty(max(ws, 256), dtype=torch.uint8, device=dev)
    stream = torch.cuda.current_stream(dev)

    def step(p=prec, o=out):
        cfd.cfd_exchange_ghosts(blocks, fields, nf, stream)
        cfd.cfd_advect(blocks, fields, nf, beta, p, n_iter, o, work, stream)

    for _ in range(args.warmup):
        step()
    cfd.cfd_sync_status(blocks, stream)
    torch.cuda.synchronize()
    clocks = ClockSampler(local)
    launches0 = cfd.cfd_kernel_launches()
    if world > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    clocks.start()
    time.sleep(0.3)
    ms_step = timed(step, args.steps, stream, torch)
    if world > 1:
        torch.distributed.barrier()
    clk = clocks.stop()
    cfd.cfd_sync_status(blocks, stream)
    launches = cfd.cfd_kernel_launches() - launches0
    prof_steps = max(3, min(args.steps, 50))
    cfd.cfd_profile_enable(True)
    torch.cuda.synchronize()
    ms_prof = timed(step, prof_steps, stream, torch)
    prof = {name: cfd.cfd_profile_read(fid) for name, fid in cfd.KERNEL_FAMILIES.items()}
    cfd.cfd_profile_enable(False)
    ms_step = max_over_ranks(ms_step, dev)
    value = whole_job_value(units, world, ms_step)

    nl, tl = prof["biased"]
    fpp = advect_flops_per_point_axis(9, n_iter, N, g) * 3
    fl = fpp * units * prof_steps
    ndl, tdl = prof["dense"]
    # pencils along each axis on which the shift changes sign need both biased solves
    mixed = []
    if not box:
        bi = beta.view(mesh.nblocks, 3, E, E, E)[:, :, g:g + N, g:g + N, g:g + N]
        for i, dim in ((0, 4), (1, 3), (2, 2)):      # beta^x along x (dim 4), beta^y along y, beta^z along z
            comp = bi[:, i]
            mixed.append(float(((comp > 0).any(dim=dim - 1) & (comp < 0).any(dim=dim - 1)).double().mean()))
    elem_f = fields.element_size()
    byts = (2 + 3 / nf) * elem_f * units * prof_steps         # f and out once, beta once for all fields
    peaks = {}
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as fh:
            peaks = json.load(fh)
    except OSError:
        pass
    hbm = float(peaks.get("hbm_gbs", 6800.0))
    if prec != cfd.CFD_FP64_BANDED:
        # k_dense: per axis the field is read once and both biased derivatives written once; each
        # halo pass of the iteration (k_halo_rows) reads the field again.  The blend kernel reads the
        # upwind derivative of each axis per field, the three shift components once per point,
        # and writes the term.
        elem = fields.element_size()
        per_pf = 3 * 3 * elem
        ach = per_pf * units * prof_steps / (tdl * 1e-3) / 1e9
        nhl, thl = prof["dense_halo"]
        comb_b = (3 + 1 + 3 / nf) * elem * units * prof_steps
        roof = {"kernel": "k_dense (tcgen05 BF16 digit-slice GEMM, biased operators D+ and D-)", "bound": "hbm",
                "achieved": round(ach, 1), "peak": hbm, "unit": "GB/s", "frac": round(ach / hbm, 4),
                "peak_source": "measured" if "hbm_gbs" in peaks else "fallback",
                "algorithmic_bytes_per_point_field": round(per_pf, 2),
                "traffic": MEASURED_TRAFFIC.get((args.workload, args.prec, n_iter)),
                "algorithmic_bytes_per_launch": round(per_pf * units / max(ndl / prof_steps, 1)),
                "launches_per_step": ndl / prof_steps, "avg_launch_ms": round(tdl / max(ndl, 1), 5),
                "share_of_step": round(tdl / (ms_prof * prof_steps), 4),
                "halo_passes": {"kernel": "k_halo_rows (compensated FP32 on the CUDA cores)",
                                "launches_per_step": nhl / prof_steps, "ms_per_step": round(thl / prof_steps, 4),
                                "hbm_gbs": round(3 * n_iter * elem * units * prof_steps / (thl * 1e-3) / 1e9, 1)
                                if thl > 0 else None},
                "blend": {"kernel": "k_advect_combine", "launches_per_step": nl / prof_steps,
                          "ms_per_step": round(tl / prof_steps, 4),
                          "hbm_gbs": round(comb_b / (tl * 1e-3) / 1e9, 1) if tl > 0 else None},
                "events_region": {"steps": prof_steps, "ms_per_step": round(ms_prof, 5)}}
    else:
        achieved = fl / (tl * 1e-3) / 1e9
        roof = {"kernel": "k_biased (FP64 upwind bidiagonal pencil solves)", "bound": "alu",
                "achieved": round(achieved, 2), "peak": FP64_NOMINAL_GFLOPS, "unit": "GFLOP/s",
                "frac": round(achieved / FP64_NOMINAL_GFLOPS, 4),
                "peak_source": "FP64 nominal 1.25 TFLOP/s (profiling recipe table)",
                "flops_per_point_field": round(fpp, 2),
                "flops_definition": "upwind side only: 2 taps + scale + recurrence + beta product per axis, "
                                    "plus the halo rows of the non-final passes",
                "mixed_sign_pencils_xyz": [round(v, 4) for v in mixed],
                "hbm_achieved_gbs": round(byts / (tl * 1e-3) / 1e9, 1), "hbm_peak_gbs": hbm,
                "algorithmic_bytes_per_point_field": round((2 + 3 / nf) * elem_f, 2),
                "traffic": MEASURED_TRAFFIC.get((args.workload, args.prec, n_iter)),
                "launches_per_step": nl / prof_steps, "avg_launch_ms": round(tl / max(nl, 1), 5),
                "share_of_step": round(tl / (ms_prof * prof_steps), 4),
                "events_region": {"steps": prof_steps, "ms_per_step": round(ms_prof, 5)}}

    compare = None
    if not args.no_compare and prec != cfd.CFD_FP64_BANDED:
        ref = torch.empty_like(out)
        step(cfd.CFD_FP64_BANDED, ref)
        torch.cuda.synchronize()
        ms64 = timed(lambda: step(cfd.CFD_FP64_BANDED, ref), args.compare_steps, stream, torch)
        step()
        torch.cuda.synchronize()
        err = (out.double() - ref.double()).abs().max()
        rel = [float(err / ref.double().abs().max())]
        compare = {"fp64_banded": {"value": round(units / (ms64 * 1e-3) / 1e9, 4), "ms_per_step": round(ms64, 4)},
                   "speedup_vs_fp64_banded": round(ms64 / ms_step, 3), "max_rel_err_vs_fp64_banded": max(rel)}
        del ref

    e2e = None
    if not args.no_e2e:
        host_in = torch.empty(fields.numel(), dtype=fields.dtype, pin_memory=True)
        host_in.copy_(fields)
        host_out = torch.empty(out.numel(), dtype=out.dtype, pin_memory=True)

        def step_e2e():
            fields.copy_(host_in, non_blocking=True)
            step()
            host_out.copy_(out, non_blocking=True)

        step_e2e()
        torch.cuda.synchronize()
        ms_e2e = timed(step_e2e, max(3, min(20, args.steps // 10)), stream, torch)
        e2e = {"value": round(units * world / (ms_e2e * 1e-3) / 1e9, 4), "unit": "Gpoint-ops/s",
               "h2d_bytes_per_step": host_in.numel() * host_in.element_size(),
               "d2h_bytes_per_step": host_out.numel() * host_out.element_size(), "ms_per_step": round(ms_e2e, 4)}
    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        cpu = cpu_baseline(spec)
    if rank == 0:
        in_bytes = fields.numel() * fields.element_size()
        line = {
            "metric": ADVECT_METRIC, "value": round(value, 4),
            "unit": "Gpoint-ops/s", "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": round(ms_step, 5), "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": spec["dtype"], "data": "synthetic (seeded analytic fields and shift)",
            "config": {"workload": args.workload, "path": args.prec, "n_iter": n_iter, "fields": nf,
                       "blocks": mesh.nblocks, "points_per_field": nint,
                       "l2": "inputs larger than L2" if in_bytes > L2_BYTES else "inputs fit L2",
                       "input_bytes": in_bytes, "parallelism": f"replicas x{world}"},
            "roofline": roof, "compare": compare, "cpu_baseline": cpu, "e2e": e2e, "gpu_launches": int(launches),
            "clocks": clk,
        }
        print(json.dumps(line))
    if world > 1:
        torch.distributed.destroy_process_group()


def adv2d_profile(x, y):
    """u(x, y) = g(x) h(y) of Sec. "Two dimensional advection": g of Eq. test_grid_conv_g with
    (A, x0, N1, S) = (5/100, 2/10, 2, 1), h of Eq. test_grid_conv_h with
    (S, x0, c1, c2, N1, N2, phi_S) = (15/10, pi, 12/10, -1, 2, 7, 1); works on numpy or torch."""
    lib = np if isinstance(x, np.ndarray) else __import__("torch")
    gx = 0.05 * lib.exp(-1.0 * lib.sin(2 * (x - 0.2)))
    hy = lib.exp(-1.5 * (y - math.pi) ** 2) * (1.2 * lib.sin(7 * y) - lib.cos(7 * y)) + lib.sin(2 * y - 1.0)
    return gx * hy


def run_adv2d(args, spec):
    """2D advection on the GPU: steps/s, Gpoint-ops/s (points x 4 stages, one advective term each)
    and the max error against the exactly translated profile after the timed steps."""
    import torch
    from paper_2302_14858_gb300 import cfd, workloads as W
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl")
    dev = torch.device("cuda", local)
    torch.cuda.set_device(dev)
    NM, N, g = spec["NM"], spec["N"], 4
    nb = NM // N
    mesh = W.periodic_box_mesh(nb, nb, 1, N, g)
    E = N + 2 * g
    dx = 2 * math.pi / NM
    phi = math.radians(spec["angle_deg"])
    c = (math.cos(phi), math.sin(phi))
    dt = spec["cfl"] * dx
    coef = ([0.0, 0.068841064670197562, 0.62754761399692844, -0.59911219706265022],
            [1.0, 0.81058824734452378, 1.3891900984667538, 1.2610225117075399],
            [1.2299693289723146, 0.079894519849001553, 0.93225854169045408, 0.45482163406909008],
            [1.0, 0.14874467817694941, -0.88063710498437737, 1.0])

    def field(t):
        # interior and ghosts of every block from the translated profile, periodic in x and y
        out = torch.empty((mesh.nblocks, E, E, E), dtype=torch.float64, device=dev)
        loc = (torch.arange(-g, N + g, dtype=torch.float64, device=dev) + 0.5)
        for b in range(mesh.nblocks):
            xs = (mesh.origin[b, 0] + loc) * dx
            ys = (mesh.origin[b, 1] + loc) * dx
            Y, X = torch.meshgrid(ys, xs, indexing="ij")
            u = adv2d_profile(torch.remainder(X - c[0] * t, 2 * math.pi), torch.remainder(Y - c[1] * t, 2 * math.pi))
            out[b] = u[None, :, :].expand(E, E, E)
        return out.reshape(-1)

    u0 = field(0.0)
    u = u0.clone()
    beta = torch.empty((mesh.nblocks, 3, E, E, E), dtype=torch.float64, device=dev)
    beta[:, 0] = -c[0]
    beta[:, 1] = -c[1]
    beta[:, 2] = 0.0
    beta = beta.reshape(-1)
    d1, _ = scheme_descs()
    scheme = cfd.cfd_scheme_create(d1, None)
    cfd.cfd_scheme_set_biased(scheme, biased_desc())
    blocks = cfd.cfd_blocks_bind(scheme, mesh.n, mesh.dx, mesh.neighbors, g, cfd.CFD_F64)
    stream = torch.cuda.current_stream(dev)
    n_iter = spec["n_iter"]
    sigma, r = 0.04, 4

    def run(prec, steps, graph=False):
        work = torch.empty(cfd.cfd_advect_lsrk_workspace(blocks, 1, prec, n_iter), dtype=torch.uint8, device=dev)
        step = lambda st=stream: cfd.cfd_advect_lsrk_step(blocks, u, 1, beta, dt, coef, sigma, r, prec, n_iter,
                                                          work, st)
        u.copy_(u0)
        for _ in range(args.warmup):
            step()
        u.copy_(u0)
        torch.cuda.synchronize()
        if graph:
            # G steps captured once into a CUDA graph (the launches of a small problem dominate)
            G = 10
            side = torch.cuda.Stream(dev)
            side.wait_stream(stream)
            gr = torch.cuda.CUDAGraph()
            with torch.cuda.graph(gr, stream=side):
                cur = torch.cuda.current_stream(dev)
                for _ in range(G):
                    step(cur)
            stream.wait_stream(side)
            u.copy_(u0)
            torch.cuda.synchronize()
            reps = max(1, steps // G)
            ms = timed(gr.replay, reps, torch.cuda.current_stream(dev), torch) / G
            steps = reps * G
        else:
            ms = timed(step, steps, stream, torch)
        cfd.cfd_sync_status(blocks, stream)
        exact = field(steps * dt).view(mesh.nblocks, E, E, E)[:, g:g + N, g:g + N, g:g + N]
        got = u.view(mesh.nblocks, E, E, E)[:, g:g + N, g:g + N, g:g + N]
        err = float((got - exact).abs().max())
        return ms, err

    prec = PREC[args.prec]
    clocks = ClockSampler(local)
    launches0 = cfd.cfd_kernel_launches()
    clocks.start()
    time.sleep(0.3)
    ms, err = run(prec, args.steps)
    clk = clocks.stop()
    launches = cfd.cfd_kernel_launches() - launches0
    ms = max_over_ranks(ms, dev)
    units = NM * NM * N * 4
    compare = None
    if not args.no_compare and prec != PREC["fp64_banded"]:
        ms64, err64 = run(PREC["fp64_banded"], args.steps)
        compare = {"fp64_banded": {"steps_per_s": round(1e3 / ms64, 3), "ms_per_step": round(ms64, 4),
                                   "max_err_vs_exact": err64}, "speedup_vs_fp64_banded": round(ms64 / ms, 3)}
    graph = None
    if args.graph:
        msg, errg = run(prec, args.steps, graph=True)
        graph = {"steps_per_s": round(1e3 / msg, 3), "ms_per_step": round(msg, 5), "max_err_vs_exact": errg,
                 "value": round(whole_job_value(units, world, msg), 4), "steps_per_graph": 10}
    cpu = cpu_baseline(spec) if (rank == 0 and world == 1 and not args.no_cpu_baseline) else None
    if rank == 0:
        line = {
            "metric": ADV2D_METRIC, "value":
                round(whole_job_value(units, world, ms), 4), "unit": "Gpoint-ops/s", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(ms, 5), "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic (the paper's analytic profile g(x) h(y))",
            "config": {"workload": args.workload, "path": args.prec, "n_iter": n_iter, "blocks": mesh.nblocks,
                       "grid": [NM, NM], "block": N, "angle_deg": spec["angle_deg"], "cfl": spec["cfl"],
                       "ko": {"sigma": sigma, "r": r}, "parallelism": f"replicas x{world}"},
            "steps_per_s": round(1e3 / ms * world, 3), "t_final": args.steps * dt, "max_err_vs_exact": err,
            "compare": compare, "graph": graph, "cpu_baseline": cpu, "gpu_launches": int(launches), "clocks": clk,
        }
        print(json.dumps(line))
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


def run_wave(args, spec):
    """The RK4 wave driver: Gpoint-ops/s (3 second-derivative ops x points x 4 stages per step),
    steps/s, and the phase and amplitude errors of every plane-wave mode against the exact
    solution after the timed steps (both the requested path and the FP64 banded path)."""
    import torch
    from paper_2302_14858_gb300 import cfd, workloads as W
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl")
    dev = torch.device("cuda", local)
    torch.cuda.set_device(dev)
    NM, N, g = spec["NM"], spec["N"], 4
    mesh = W.uniform_mesh(NM, N, g)
    nb, E = NM // N, N + 2 * g
    dx = 2 * math.pi / NM
    dt = 0.25 * dx
    pw = W.plane_waves(2302 + 5, spec["modes"], spec["kmax"])
    x = (torch.arange(NM, dtype=torch.float64, device=dev) + 0.5) * dx
    idx = (torch.arange(nb, device=dev)[:, None] * N + torch.arange(-g, N + g, device=dev)[None, :]) % NM

    def layout(fg):
        ext = fg[idx[:, None, None, :, None, None], idx[None, :, None, None, :, None], idx[None, None, :, None, None, :]]
        return ext.reshape(-1).contiguous()

    def plane(t, deriv):
        Z, Y, X = torch.meshgrid(x, x, x, indexing="ij")
        out = torch.zeros_like(X)
        for kv, A, p in zip(pw.k, pw.A, pw.phi):
            w = float(np.sqrt((kv ** 2).sum()))
            arg = float(kv[0]) * X + float(kv[1]) * Y + float(kv[2]) * Z - w * t + float(p)
            out += float(A) * (w * torch.sin(arg) if deriv else torch.cos(arg))
        return out

    phi0, K0 = layout(plane(0.0, False)), layout(plane(0.0, True))
    d1, d2 = scheme_descs()
    scheme = cfd.cfd_scheme_create(d1, d2)
    shift = spec.get("shift")
    if shift is not None:
        cfd.cfd_scheme_set_biased(scheme, biased_desc())
        beta = torch.empty((mesh.nblocks, 3, E, E, E), dtype=torch.float64, device=dev)
        for i, v in enumerate(shift):
            beta[:, i] = float(v)
        beta = beta.reshape(-1)
    blocks = cfd.cfd_blocks_bind(scheme, mesh.n, mesh.dx, mesh.neighbors, g, cfd.CFD_F64)
    stream = torch.cuda.current_stream(dev)
    phi, K = phi0.clone(), K0.clone()

    lsrk = args.integrator == "lsrk2s" or shift is not None
    if lsrk:
        # a 4-stage 4th-order member of the 2S family (coefficients solved from the order conditions)
        coef = ([0.0, 0.068841064670197562, 0.62754761399692844, -0.59911219706265022],
                [1.0, 0.81058824734452378, 1.3891900984667538, 1.2610225117075399],
                [1.2299693289723146, 0.079894519849001553, 0.93225854169045408, 0.45482163406909008],
                [1.0, 0.14874467817694941, -0.88063710498437737, 1.0])

    def one_step(prec, work):
        if shift is not None:
            cfd.cfd_shifted_wave_lsrk_step(blocks, phi, K, beta, dt, coef, args.sigma, args.ko_r, prec, spec["n_iter"],
                                           work, stream)
        elif lsrk:
            cfd.cfd_wave_lsrk_step(blocks, phi, K, dt, coef, args.sigma, args.ko_r, prec, spec["n_iter"], work, stream)
        else:
            cfd.cfd_wave_rk_step(blocks, phi, K, dt, prec, spec["n_iter"], work, stream)

    def run(prec, steps, timed_region):
        ws = (cfd.cfd_shifted_wave_workspace if shift is not None else
              cfd.cfd_wave_lsrk_workspace if lsrk else cfd.cfd_wave_workspace)(blocks, prec, spec["n_iter"])
        work = torch.empty(ws, dtype=torch.uint8, device=dev)
        phi.copy_(phi0)
        K.copy_(K0)
        for _ in range(args.warmup):
            one_step(prec, work)
        phi.copy_(phi0)
        K.copy_(K0)
        torch.cuda.synchronize()
        ms = timed(lambda: one_step(prec, work), steps, stream, torch) if timed_region else None
        if not timed_region:
            for _ in range(steps):
                one_step(prec, work)
            torch.cuda.synchronize()
        cfd.cfd_sync_status(blocks, stream)
        return ms, mode_errors(steps * dt)

    def mode_errors(t):
        # interior values back to the global grid, then project on every plane-wave mode
        f = phi.view(nb, nb, nb, E, E, E)[:, :, :, g:g + N, g:g + N, g:g + N]
        fg = f.permute(0, 3, 1, 4, 2, 5).reshape(NM, NM, NM)
        Z, Y, X = torch.meshgrid(x, x, x, indexing="ij")
        amp, ph = 0.0, 0.0
        for kv, A, p in zip(pw.k, pw.A, pw.phi):
            w = float(np.sqrt((kv ** 2).sum()))
            if shift is not None:                    # shifted system: frequency |k| - beta.k
                w -= float(sum(float(b) * float(kk) for b, kk in zip(shift, kv)))
            arg = float(kv[0]) * X + float(kv[1]) * Y + float(kv[2]) * Z
            c = complex((fg * torch.cos(arg)).mean().item() * 2.0, -(fg * torch.sin(arg)).mean().item() * 2.0)
            want = float(A) * complex(math.cos(float(p) - w * t), math.sin(float(p) - w * t))
            r = c / want
            amp = max(amp, abs(abs(r) - 1.0))
            ph = max(ph, abs(math.atan2(r.imag, r.real)))
        return {"amplitude_err_max": amp, "phase_err_max_rad": ph}

    prec = PREC[args.prec]
    clocks = ClockSampler(local)
    launches0 = cfd.cfd_kernel_launches()
    clocks.start()
    time.sleep(0.3)
    ms, err = run(prec, args.steps, True)
    clk = clocks.stop()
    launches = cfd.cfd_kernel_launches() - launches0
    ms = max_over_ranks(ms, dev)
    # 3 second-derivative ops per point and stage (+ the two upwinded advective terms when shifted)
    units = (3 + (2 if shift is not None else 0)) * NM ** 3 * 4
    cpu = cpu_baseline(spec) if (rank == 0 and world == 1 and not args.no_cpu_baseline) else None
    compare = None
    if not args.no_compare and prec != PREC["fp64_banded"]:
        ms64, err64 = run(PREC["fp64_banded"], args.steps, True)
        compare = {"fp64_banded": {"value": round(units / (ms64 * 1e-3) / 1e9, 4), "ms_per_step": round(ms64, 4),
                                   **err64},
                   "speedup_vs_fp64_banded": round(ms64 / ms, 3)}
    if rank == 0:
        line = {
            "metric": METRIC, "value": round(whole_job_value(units, world, ms), 4), "unit": "Gpoint-ops/s",
            "n_gpus": world, "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(ms, 5),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic (seeded plane waves)",
            "config": {"workload": args.workload, "path": args.prec, "n_iter": spec["n_iter"], "blocks": mesh.nblocks,
                       "dt_over_dx": 0.25, "modes": spec["modes"], "kmax": spec["kmax"],
                       "integrator": "lsrk2s" if lsrk else args.integrator,
                       "ko": {"sigma": args.sigma, "r": args.ko_r} if lsrk else None,
                       "shift": list(shift) if shift is not None else None,
                       "l2": "inputs larger than L2", "parallelism": f"replicas x{world}"},
            "steps_per_s": round(1e3 / ms * world, 3), "t_final": args.steps * dt, **err,
            "compare": compare, "cpu_baseline": cpu, "gpu_launches": int(launches), "clocks": clk,
        }
        print(json.dumps(line))
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


def run_reference(args, spec, rank):
    """The oracle as the reference arm, on host cores, same metric and config."""
    if rank != 0:
        return
    pool = OraclePool(spec) if spec["kind"] in ("uniform", "boxinbox") else None
    one = (lambda sec: pool.run(sec)) if pool else (lambda sec: cpu_baseline(spec, seconds=sec))
    try:
        for _ in range(args.warmup):
            one(0.5)
        vals = []
        t0 = time.perf_counter()
        for _ in range(args.steps):
            vals.append(one(2.0))
        el = time.perf_counter() - t0
    finally:
        if pool:
            pool.close()
    v = statistics.median(r["value"] for r in vals)
    metric = {"advect": ADVECT_METRIC, "adv2d": ADV2D_METRIC}.get(spec["kind"], METRIC)
    line = {"metric": metric, "value": round(v, 6),
            "unit": "Gpoint-ops/s", "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(el / args.steps * 1e3, 3),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic (seeded analytic fields)", "impl": "reference",
            "config": {"workload": args.workload, "path": "oracle (numpy FP64, host)", "n_iter": spec["n_iter"]},
            "cpu_baseline": {"value": round(v, 6), "unit": "Gpoint-ops/s", "cores": vals[0]["cores"], "kind": "oracle",
                             "sample": vals[0]["sample"]},
            "e2e": {"value": round(v, 6), "unit": "Gpoint-ops/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line))


if __name__ == "__main__":
    main()
