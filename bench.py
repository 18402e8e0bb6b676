"""Throughput of the two-step Brillouin-zone propagation on GB300.

Workload (one "step" = one full time step of every sub-simulation): the
two-step linear-response run of 64 shifted 4^3 Monkhorst-Pack subgrids of
the 8-atom cubic Si-like cell (a = 10.26 bohr, 16^3 grid, 16 doubly
occupied bands, 32 KB projectors), i.e. 4096 k-points and 65 536 orbitals,
kick 0.005 along x, dt = 0.08, 4th-order Taylor, self-consistent v_Hxc.
Inputs are synthetic (plane-wave start orbitals) and larger than L2.

metric: orbital-steps/s = (k, band, dt) units advanced per second.
  value : FP32/tensor-path throughput, device-resident inputs, CUDA events
  e2e   : the same through the C ABI with host buffers (ground-state upload,
          propagation, current download inside the timed region)
  fp64  : the plain FP64 GPU path on the same workload (context)

--impl reference times the CPU oracle (the reference of this build) on
host cores, one bounded sample of the workload per step.
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

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)
# The oracle's worker processes re-import this module: one BLAS thread each.
os.environ.setdefault("OPENBLAS_NUM_THREADS", "1")
os.environ.setdefault("OMP_NUM_THREADS", "1")

import numpy as np  # noqa: E402

METRIC = "orbital-steps/s (k·band·Δt), FP32/TC batched vs FP64 GPU; ε(ω) rel err vs oracle"
UNIT = "orbital-steps/s"
WORKLOAD = "two-step 64x4^3 shifted MP, Si-like 8-atom cubic cell, 16^3 grid, 16 bands (one time step)"


# ----------------------------------------------------------------------------
# CPU oracle timing (reference arm and cpu_baseline)
# ----------------------------------------------------------------------------
def _oracle_worker(conn, m, max_steps):
    """One host process holding one sub-simulation of the two-step workload
    (shifted 4^3 subgrid m: 64 k-points x 16 bands, plane-wave start, kick).
    Commands: ("step", n) propagates n time steps with the oracle and returns
    (propagate-only seconds, orbital-steps); ("quit", 0) ends the process.
    The oracle's propagate() also evaluates rho, v_Hxc, J(0-) and J(0+) of its
    start state; that fixed part is measured once (a call with no steps) and
    subtracted, so the returned time is that of the time steps alone."""
    import workloads as W
    from oracle import dynamics, kpoints
    run = W.twostep_kick_run(n_steps=max_steps)
    sub = run.subsims[m % len(run.subsims)]
    cell = sub.cell
    nk = sub.mp[0] * sub.mp[1] * sub.mp[2]
    u = W.plane_wave_orbitals(cell.a, cell.n, W.plane_wave_set(cell.n_bands), nk)
    k = kpoints.kpoints_cartesian(cell.a, sub.mp, sub.shift)
    ops = dynamics.Operators(cell)
    a_all = dynamics.field_samples(sub.field, sub.dt, max_steps)
    fixed = []
    for _ in range(2):
        t0 = time.perf_counter()
        dynamics.propagate(cell, k, u, sub.dt, 0, a_all[:1], ops=ops, keep_state=False)
        fixed.append(time.perf_counter() - t0)
    t_fixed = min(fixed)
    step = 0
    conn.send(("ready", t_fixed))
    while True:
        cmd, n = conn.recv()
        if cmd != "step":
            break
        t0 = time.perf_counter()
        res = dynamics.propagate(cell, k, u, sub.dt, n, a_all[2 * step: 2 * (step + n) + 1], ops=ops)
        dt_wall = time.perf_counter() - t0
        u = res["u"]
        step += n
        conn.send((max(dt_wall - t_fixed, 1e-9), nk * cell.n_bands * n))
    conn.close()


class OraclePool:
    """`workers` host processes, one sub-simulation each (spawned, one BLAS
    thread per process), stepped together: the CPU oracle timed on a bounded
    sample of the benchmark workload."""

    def __init__(self, workers: int, max_steps: int):
        import multiprocessing as mp
        ctx = mp.get_context("spawn")
        self.conns, self.procs = [], []
        for m in range(workers):
            a, b = ctx.Pipe()
            p = ctx.Process(target=_oracle_worker, args=(b, m, max_steps), daemon=True)
            p.start()
            self.conns.append(a)
            self.procs.append(p)
        self.t_fixed = [c.recv()[1] for c in self.conns]

    def step(self, n: int = 1):
        """All workers advance n steps at once; returns (orbital-steps, wall
        seconds of the parallel step = the slowest worker's propagate time)."""
        for c in self.conns:
            c.send(("step", n))
        res = [c.recv() for c in self.conns]
        return sum(r[1] for r in res), max(r[0] for r in res)

    def close(self):
        for c in self.conns:
            try:
                c.send(("quit", 0))
            except (BrokenPipeError, OSError):
                pass
        for p in self.procs:
            p.join(timeout=30)


def oracle_baseline(workers: int, steps: int, warmup: int = 1):
    """cpu_baseline: `workers` processes (one per host core) x `steps` timed
    time steps after `warmup`, then one process alone for a 1-core figure."""
    pool = OraclePool(workers, warmup + steps)
    try:
        if warmup:
            pool.step(warmup)
        units, wall = pool.step(steps)
    finally:
        pool.close()
    one = OraclePool(1, 2)
    try:
        one.step(1)
        u1, w1 = one.step(1)
    finally:
        one.close()
    return units / wall, units, wall, u1 / w1


def host_cores() -> int:
    try:
        return len(os.sched_getaffinity(0))
    except AttributeError:
        return os.cpu_count() or 1


def cpu_model() -> str:
    try:
        with open("/proc/cpuinfo") as f:
            for line in f:
                if line.lower().startswith(("model name", "cpu part")):
                    return line.split(":", 1)[1].strip()
    except OSError:
        pass
    return "unknown"


# ----------------------------------------------------------------------------
# Clocks
# ----------------------------------------------------------------------------
class ClockSampler:
    """SM clock and clock-event reasons sampled during the timed region.

    NVML (libnvidia-ml through ctypes, read-only queries) every 10 ms when it
    loads, so that even a short timed region gets many samples; otherwise
    nvidia-smi every 100 ms.  The GPU is found by the UUID CUDA reports for
    this process's device, falling back to the device index."""
    Q = ("clocks.sm,clocks.max.sm,clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
    # clock-event reason bits of nvmlDeviceGetCurrentClocksEventReasons
    BITS = {"sw_power_cap": 0x4, "hw_slowdown": 0x8, "sw_thermal_slowdown": 0x20, "hw_thermal_slowdown": 0x40}

    def __init__(self, index: int = 0, uuid: str | None = None):
        self.index = index
        self.uuid = uuid
        self.proc = None
        self.nvml = None
        self.stop = threading.Event()
        self.samples = []   # (sm_mhz, max_mhz, set of reasons)
        self.source = None

    def _nvml_open(self):
        import ctypes
        lib = ctypes.CDLL("libnvidia-ml.so.1")
        if lib.nvmlInit_v2() != 0:
            return None
        h = ctypes.c_void_p()
        ok = False
        if self.uuid:
            for u in (self.uuid, "GPU-" + self.uuid):
                if lib.nvmlDeviceGetHandleByUUID(u.encode(), ctypes.byref(h)) == 0:
                    ok = True
                    break
        if not ok:
            ok = lib.nvmlDeviceGetHandleByIndex_v2(ctypes.c_uint(self.index), ctypes.byref(h)) == 0
        if not ok:
            lib.nvmlShutdown()
            return None
        reasons = getattr(lib, "nvmlDeviceGetCurrentClocksEventReasons", None) or \
            lib.nvmlDeviceGetCurrentClocksThrottleReasons
        return lib, h, reasons

    def _nvml_loop(self):
        import ctypes
        lib, h, reasons = self.nvml
        clk, mx, rs = ctypes.c_uint(), ctypes.c_uint(), ctypes.c_ulonglong()
        while not self.stop.is_set():
            if (lib.nvmlDeviceGetClockInfo(h, 1, ctypes.byref(clk)) == 0 and
                    lib.nvmlDeviceGetMaxClockInfo(h, 1, ctypes.byref(mx)) == 0 and
                    reasons(h, ctypes.byref(rs)) == 0):
                act = {nm for nm, b in self.BITS.items() if rs.value & b}
                self.samples.append((float(clk.value), float(mx.value), act))
            self.stop.wait(0.01)

    def __enter__(self):
        try:
            self.nvml = self._nvml_open()
        except (OSError, AttributeError):
            self.nvml = None
        if self.nvml:
            self.source = "nvml 10 ms"
            self.thread = threading.Thread(target=self._nvml_loop, daemon=True)
            self.thread.start()
            return self
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.Q}",
                                          "--format=csv,noheader,nounits", "-lms", "100"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.source = "nvidia-smi 100 ms"
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except (OSError, FileNotFoundError):
            self.proc = None
        return self

    def _read(self):
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in self.proc.stdout:
            parts = [p.strip() for p in line.strip().split(",")]
            if len(parts) < 6:
                continue
            try:
                sm, mx = float(parts[0]), float(parts[1])
            except ValueError:
                continue
            self.samples.append((sm, mx, {nm for nm, v in zip(names, parts[2:6]) if v.lower() == "active"}))

    def __exit__(self, *a):
        self.stop.set()
        if self.nvml:
            self.thread.join(timeout=2)
            self.nvml[0].nvmlShutdown()
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self):
        if not self.samples:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"]}
        reasons = set()
        for _, _, r in self.samples:
            reasons |= r
        return {"sm_mhz": statistics.median(x[0] for x in self.samples),
                "sm_max_mhz": max(x[1] for x in self.samples), "reasons": sorted(reasons),
                "samples": len(self.samples), "source": self.source}


def device_uuid(index: int) -> str | None:
    import torch
    try:
        u = getattr(torch.cuda.get_device_properties(index), "uuid", None)
        return str(u) if u is not None else None
    except Exception:
        return None


# ----------------------------------------------------------------------------
# GPU arm
# ----------------------------------------------------------------------------
def benchmark_run(n_steps_cap, world=1, n_subsims=64):
    """The benchmark's sub-simulations over `world` ranks (weak scaling: 64 per
    rank).  Block 0 is the two-step run of 64 lattice-shifted 4^3 subgrids of
    the 16^3 Monkhorst-Pack grid (Eq. 10); block j >= 1 is the same set with
    every shift moved by h_j / 4, h_j the j-th Halton point (bases 2, 3, 5), i.e.
    a 16^3 grid displaced by a fraction h_j of its spacing, so that the blocks
    together form one larger two-step sample (Eq. 9)."""
    import dataclasses
    import workloads as W
    from paper_2112_00920_gb300 import halton
    run = W.twostep_kick_run(n_steps=n_steps_cap)
    base = run.subsims[:n_subsims]
    subs = list(base)
    if world > 1:
        h = np.asarray(halton(world - 1)).reshape(world - 1, 3)
        for j in range(1, world):
            subs += [dataclasses.replace(sp, shift=tuple(float(v) for v in np.asarray(sp.shift) + h[j - 1] / 4.0))
                     for sp in base]
    run.subsims = subs
    return run


def build_propagator(precision, n_steps_cap, device=0, n_subsims=64, block=None, world=1):
    from paper_2112_00920_gb300 import Propagator, shifted_kpoints
    run = benchmark_run(n_steps_cap, world, n_subsims)
    run.subsims = run.subsims[block[0]:block[1]] if block is not None else run.subsims[:n_subsims]
    cell = run.subsims[0].cell
    P = Propagator(precision, device=device)
    cid = P.add_cell_spec(cell)
    sids = [P.add_subsim(cid, shifted_kpoints(cell.a, s.mp, s.shift), s.dt, n_steps_cap) for s in run.subsims]
    return P, sids, run


STAGE_KERNEL = {
    "fp32": "k_stage_fused (z-march stencil + tensor-core projector contractions + Taylor accumulate), one launch "
            "per Taylor stage",
    "fp32_tc": "k_stage_zb (z-march stencil + non-local term + Taylor accumulate)",
    "fp64": "k_stage (stencil + ket + Taylor accumulate)",
}
STEP_KERNEL = ("k_step_fused (the four Taylor stages of a time step in one launch: z-march stencil, tensor-core "
               "projector z contractions (tcgen05 + TMEM in variant 0, mma.sync in variant 3), Taylor "
               "accumulation in registers)")
# FP32 arithmetic of the local part of h, the Taylor scaling and the psi sum,
# per grid point, orbital and Taylor stage (complex values): Laplacian and
# gradient pairs 3 axes x 4 x (2 + 4 + 2 + 4) = 144, q.grad 10, diagonal 3,
# combination 4, (-i dt/m) 2, accumulation 2.
FLOPS_LOCAL_PER_POINT_STAGE = 165
FP32_LANES_PER_SM = 128
# DRAM bytes of one k_step_fused launch from an ncu capture (dram__bytes_read.sum
# + dram__bytes_write.sum) on the reduced workload (8 of the 64 subgrids, 8192
# orbitals), scaled by the orbital count to the full workload.  Valid only for
# the source it was taken on: the SHA-1 of the kernel header is checked at run time.
STEP_TRAFFIC = {"file": "tsbz_fused.cuh", "sha1": "93d95614680d5daa93a0a54a1c9dbb337bade2aa",
                "bytes_per_launch_full": 8 * (273.970432e6 + 218.047744e6),
                "profile": "profiles/k_step_fused_tcgen05_twostep8.md"}
# DRAM bytes of the per-stage stencil kernel k_stage_zb<false> from an ncu capture of the
# reduced dense tensor-core workload (8 of the 64 subgrids): stages 1 and 2 moved 774.8 and
# 1295.1 MB against 805.3 and 1342.2 MB of algorithmic bytes (0.964 of them); the full
# launch is taken as that fraction of its algorithmic bytes.  Valid for the source it
# was taken on.
STENCIL_TRAFFIC = {"file": "tsbz_tc.cuh", "sha1": "2bd77934cbda428416643c624a258d0564747242",
                   "fraction_of_algorithmic": (774.778112 + 1295.140096) / (805.306368 + 1342.17728),
                   "profile": "profiles/k_stage_zb_fp32tc_twostep8.md"}


def _file_sha1(path: str) -> str | None:
    import hashlib
    try:
        return hashlib.sha1(open(path, "rb").read()).hexdigest()
    except OSError:
        return None


def alu_peaks(device):
    """Measured FMA peaks of this GPU (tsbz_probe_alu_peak), TFLOP/s, with the
    SM count and the nominal FP32 figure from the unit counts beside them."""
    import torch
    from paper_2112_00920_gb300._lib import probe_alu_peak
    props = torch.cuda.get_device_properties(device)
    out = {"sm_count": int(props.multi_processor_count)}
    for kind, iters in (("ffma", 20000), ("ffma2", 10000), ("dfma", 300)):
        f, ms = probe_alu_peak(device, kind, iters)
        out[kind + "_tflops"] = f / 1e12
        out[kind + "_ms"] = ms
    return out


def step_roofline(step_ms, n_orb, cell, elem, peaks, subsims, clocks, alu):
    """Roofline of k_step_fused.  It reads and writes psi once per step, so its
    HBM traffic is 2 arrays (plus P and Pa) and it is bound by its arithmetic
    issue, not by HBM: the ALU roofline is the primary one, against the FP32
    FMA peak measured on this GPU (the faster of the scalar and the packed
    FP32x2 FMA probe); the HBM figures are given beside it."""
    npts = cell.n_pts
    n_proj = 4 * cell.n_atoms
    flops = 4.0 * FLOPS_LOCAL_PER_POINT_STAGE * npts * n_orb
    byts = float(n_orb) * (2 * elem * npts + 6 * n_proj * elem)
    mhz = float(peaks.get("sm_max_mhz", 2070.0))
    if alu is None:   # no probe: the nominal figure from the unit counts (152 SMs)
        alu = {"sm_count": 152, "ffma_tflops": 152 * FP32_LANES_PER_SM * 2 * mhz * 1e6 / 1e12, "ffma2_tflops": 0.0}
    nominal = alu["sm_count"] * FP32_LANES_PER_SM * 2 * mhz * 1e6 / 1e12
    best = "ffma2" if alu["ffma2_tflops"] >= alu["ffma_tflops"] else "ffma"
    peak = alu[best + "_tflops"]
    achieved = flops / (step_ms / 1e3) / 1e12
    hbm = float(peaks.get("hbm_gbs", 6800.0))
    gbs = byts / (step_ms / 1e3) / 1e9
    traffic = None
    path = os.path.join(ROOT, "paper_2112_00920_gb300", "csrc", STEP_TRAFFIC["file"])
    if subsims == 64 and STEP_TRAFFIC["sha1"] and _file_sha1(path) == STEP_TRAFFIC["sha1"]:
        traffic = STEP_TRAFFIC["bytes_per_launch_full"]
    return {"kernel": STEP_KERNEL, "bound": "alu", "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
            "frac": achieved / peak, "traffic": traffic, "algorithmic_flops_per_launch": flops,
            "algorithmic_bytes_per_launch": byts,
            "peak_source": f"measured on this GPU: {best.upper()} probe (tsbz_probe_alu_peak), "
                           f"{alu['sm_count']} SMs; nominal {alu['sm_count']} SMs x {FP32_LANES_PER_SM} FP32 "
                           f"lanes x 2 flop x {mhz:.0f} MHz = {nominal:.1f} TFLOP/s",
            "alu_peaks_measured": alu,
            "launches_per_step": 1,
            "hbm": {"achieved": gbs, "peak": hbm, "unit": "GB/s", "frac": gbs / hbm,
                    "peak_source": "MEASURED_PEAKS.json hbm_gbs (burst copy)"},
            "sm_mhz_median": clocks.get("sm_mhz")}


def eps_check(precision, device):
    """Relative eps(omega) error of `precision` against the FP64 GPU path on a
    small linear-response run (see the call site)."""
    import workloads as W
    from paper_2112_00920_gb300 import Propagator, shifted_kpoints
    cell = W.cell_a()
    n, dt, k0 = 600, 0.08, 0.005
    k = shifted_kpoints(cell.a, (2, 2, 2), (0.0, 0.0, 0.0))
    psi = W.plane_wave_orbitals(cell.a, cell.n, W.plane_wave_set(cell.n_bands), 8)
    om = np.linspace(0.1, 20.0, 400) / 27.211386245988
    t = np.arange(n + 1) * dt
    win = 1.0 - 3.0 * (t / t[-1]) ** 2 + 2.0 * (t / t[-1]) ** 3
    wts = np.ones(n + 1)
    wts[0] = wts[-1] = 0.5
    out = {}
    for prec in ("fp64", precision):
        P = Propagator(prec, device=device)
        cid = P.add_cell_spec(cell)
        sid = P.add_subsim(cid, k, dt, n)
        P.load_ground_state(sid, psi)
        P.set_kick(sid, k0, (1.0, 0.0, 0.0))
        P.propagate(n)
        J, j0 = P.current(sid)
        P.close()
        dj = (J - j0[None, :])[:, 0]
        sig = dt * np.exp(1j * np.outer(om, t)) @ (wts * win * dj) / k0
        out[prec] = 1.0 + 4.0j * np.pi * sig / om
    return float(np.max(np.abs(out[precision] - out["fp64"])) / np.max(np.abs(out["fp64"])))


def stage_bytes_per_launch(elem: int, n_orb: int, npts: int, reads_v: bool = False) -> float:
    """Algorithmic DRAM bytes of the Taylor stage kernel, averaged over its
    four launches per step: m=1 reads t0 and writes t1 (2 arrays), m=2 and
    m=3 read t, read and write psi and write t (4 arrays), m=4 reads t and
    reads and writes psi (3 arrays): 13 arrays / 4 launches.  A stage kernel
    that takes the non-local term V = V_NL t_{m-1} as an input array (the
    dense tensor-core mode) also reads V in each launch: 17 arrays / 4."""
    return (17.0 if reads_v else 13.0) / 4.0 * elem * n_orb * npts


def stencil_roofline(device, n_subsims, hbm, peaks_src, steps=3):
    """HBM roofline of the per-stage stencil kernel (stencil + local potential
    + non-local input + Taylor accumulation, one launch per Taylor stage): the
    dense tensor-core mode on the benchmark workload, whose stage kernel
    (k_stage_zb) reads t_{m-1} and V and writes t_m and psi.  Events on the
    launching stream around every stage launch (tsbz_get_timings)."""
    import torch
    import workloads as W
    # step budget: one step, then per variant one untimed and `steps` timed steps
    P, sids, run = build_propagator("fp32_tc", 2 + 3 * (steps + 1), device=device, n_subsims=n_subsims)
    cell = run.subsims[0].cell
    psi = torch.from_numpy(W.plane_wave_orbitals(cell.a, cell.n, W.plane_wave_set(cell.n_bands), 64)).to(
        f"cuda:{device}")
    for sid in sids:
        P.load_ground_state(sid, psi)
    del psi
    P.set_kick(-1, 0.005, (1.0, 0.0, 0.0))
    P.propagate(1)
    n_var = P.variant(0)[1]
    per_variant = []
    for v in range(n_var):
        P.set_variant(0, v)
        P.propagate(1)
        P.set_profiling(True)
        P.propagate(steps)
        fam = P.timings()
        P.set_profiling(False)
        per_variant.append(fam["stage"] / (4 * steps))
    P.close()
    best = int(np.argmin(per_variant))
    stage_ms = per_variant[best]
    byts = stage_bytes_per_launch(8, run.n_orbitals, cell.n_pts, reads_v=True)
    gbs = byts / (stage_ms / 1e3) / 1e9
    traffic = None
    path = os.path.join(ROOT, "paper_2112_00920_gb300", "csrc", STENCIL_TRAFFIC["file"])
    if best == 0 and n_subsims == 64 and _file_sha1(path) == STENCIL_TRAFFIC["sha1"]:
        traffic = STENCIL_TRAFFIC["fraction_of_algorithmic"] * byts
    names = ["k_stage_zb<false> (band of t_{m-1} bulk-copied to shared memory, V and psi read per plane)",
             "k_stage_zb<true> (bands of t_{m-1}, V and psi bulk-copied to shared memory)",
             "k_stage_zf (halo plane per z, two CTA barriers per plane)"]
    return {"kernel": names[best] + ": one Taylor stage = FD stencil + local potential + non-local term V "
                                    "(an input array) + Taylor accumulation",
            "bound": "hbm", "achieved": gbs, "peak": hbm, "unit": "GB/s", "frac": gbs / hbm, "traffic": traffic,
            "algorithmic_bytes_per_launch": byts, "ms_per_launch": stage_ms, "peak_source": peaks_src,
            "variant": best, "ms_per_launch_by_variant": dict(zip(names[:n_var], per_variant)),
            "note": "fp32_tc mode on the benchmark workload; 17 arrays of 2 GiB per 4 launches (t_{m-1} and V "
                    "read by all 4, t_m written by 3, psi read and written by 3)"}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="gb300", choices=["gb300", "reference"])
    ap.add_argument("--precision", default="fp32", choices=["fp32", "fp32_tc", "fp64"])
    ap.add_argument("--fp64-steps", type=int, default=2)
    ap.add_argument("--etrs-steps", type=int, default=3,
                    help="steps of the ETRS propagator timed on the same workload (0: skip)")
    ap.add_argument("--stencil-steps", type=int, default=3,
                    help="steps of the dense tensor-core mode timed for the per-stage stencil roofline (0: skip)")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--profile-run", action="store_true",
                    help="run only the warm-up and timed steps (for profiler launch lists and captures)")
    ap.add_argument("--variant", type=int, default=-1,
                    help="profiler runs: force this kernel variant of the cell (default: the library's default)")
    ap.add_argument("--subsims", type=int, default=64,
                    help="number of the 64 shifted subgrids to run (profiling of a reduced case)")
    ap.add_argument("--workload", default="twostep64", choices=["twostep64"] + sorted(SIDE_WORKLOADS),
                    help="twostep64: the benchmark; the others time a side workload (one JSON line, "
                         "no baselines) for the large-cell path")
    args = ap.parse_args()
    if args.workload != "twostep64":
        run_side_workload(args)
        return

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local_rank = int(os.environ.get("LOCAL_RANK", "0"))

    if args.impl == "reference":
        if rank != 0:
            return
        run_reference(args)
        return

    # CPU baseline first (before any CUDA context exists in this process)
    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        workers = host_cores()
        val, units, wall, one_core = oracle_baseline(workers, steps=2)
        cpu = {"value": val, "unit": UNIT, "cores": workers, "kind": "oracle",
               "sample": f"{workers} of the 64 sub-simulations (64 k x 16 bands each, numpy complex128, one "
                         f"process per host core, BLAS 1 thread) x 2 time steps after 1 untimed step: "
                         f"{units} orbital-steps in {wall:.1f} s of propagate time (set-up, J(0-) and "
                         f"J(0+) excluded); {cpu_model()}",
               "one_core": {"value": one_core, "unit": UNIT,
                            "sample": "1 sub-simulation x 1 time step, one process alone"}}

    import torch
    import torch.distributed as dist

    torch.cuda.set_device(local_rank)
    if world > 1:
        dist.init_process_group("nccl" if torch.cuda.is_available() else "gloo")
    import workloads as W
    from paper_2112_00920_gb300 import build_library
    build_library()

    # room for the autotuner's trial steps (undone afterwards) within the step budget
    tune_room = 5 * 3 + 1
    cap = args.warmup + 2 * args.steps + 1 + tune_room
    # weak scaling: every rank advances its own block of 64 sub-simulations (the
    # shifted subgrids are independent, Eq. 9); the ranks meet once, for the
    # final two-step average of dJ (one all-reduce after the timed region)
    from paper_2112_00920_gb300.distributed import run_sharded
    P = sids = run = cell = n_orb = psi_host = psi_dev = n_tried = None
    tuned_variant = tuned_n = tuned_ms = stream = ms = launches = fam = clk = J_avg = None

    def run_block(b, e):
        nonlocal P, sids, run, cell, n_orb, psi_host, psi_dev, n_tried
        nonlocal tuned_variant, tuned_n, tuned_ms, stream, ms, launches, fam, clk, J_avg
        P, sids, run = build_propagator(args.precision, cap, device=local_rank, n_subsims=args.subsims,
                                        block=(b, e), world=world)
        cell = run.subsims[0].cell
        n_orb = run.n_orbitals
        gints = W.plane_wave_set(cell.n_bands)
        psi_host = W.plane_wave_orbitals(cell.a, cell.n, gints, 64)
        psi_dev = torch.from_numpy(psi_host).to(f"cuda:{local_rank}")
        for sid in sids:
            P.load_ground_state(sid, psi_dev)
        P.set_kick(-1, 0.005, (1.0, 0.0, 0.0))
        P.propagate(args.warmup)
        # the autotuner picks each cell's kernel variant on this workload (trial steps undone);
        # profiler runs keep the default variant so that their launch lists hold only the timed steps
        n_tried = 0
        if not args.profile_run:
            n_tried = P.autotune(budget_ms=5000)
        elif args.variant >= 0:
            P.set_variant(0, args.variant)
        tuned_variant, tuned_n, tuned_ms = P.variant(0)
        P.propagate(1)   # first step after tuning (forms the projections if the variant changed)
        stream = torch.cuda.current_stream()
        start, end = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        P.set_profiling(True)
        l0 = P.launches()
        if world > 1:
            dist.barrier()
        torch.cuda.synchronize()
        with ClockSampler(local_rank, device_uuid(local_rank)) as clk:
            start.record(stream)
            P.propagate(args.steps)
            end.record(stream)
            torch.cuda.synchronize()
        if world > 1:
            dist.barrier()
        ms = start.elapsed_time(end)
        launches = P.launches() - l0
        fam = P.timings()
        P.set_profiling(False)
        J_avg, _ = P.current(-1)
        return J_avg * (e - b)

    n_global = args.subsims * world
    J_two_step, block = run_sharded([1.0] * n_global, run_block)
    ms_t = torch.tensor([ms], device=f"cuda:{local_rank}")
    if world > 1:
        dist.all_reduce(ms_t, op=dist.ReduceOp.MAX)
    ms_max = float(ms_t.item())
    value = n_orb * args.steps * world / (ms_max / 1e3)

    # roofline of the dominant kernel family (the Taylor stage kernel)
    import json as _json
    peaks = {}
    try:
        peaks = _json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except OSError:
        pass
    hbm = float(peaks.get("hbm_gbs", 6800.0))
    elem = 16 if args.precision == "fp64" else 8
    variant, n_var, _ = P.variant(0)
    whole = args.precision == "fp32" and variant in (0, 3) and n_var == 4
    fam_ms = {k: v / args.steps for k, v in fam.items()}
    if whole:
        # profiler runs skip the FMA probe so that their launch lists hold the step's kernels only
        alu = alu_peaks(local_rank) if not args.profile_run else None
        roof = step_roofline(fam["stage"] / args.steps, n_orb, cell, elem, peaks, args.subsims, clk.summary(), alu)
    else:
        stage_ms = fam["stage"] / (4 * args.steps)
        bytes_launch = stage_bytes_per_launch(elem, n_orb, cell.n_pts, reads_v=args.precision == "fp32_tc")
        achieved = bytes_launch / (stage_ms / 1e3) / 1e9
        roof = {"kernel": STAGE_KERNEL[args.precision], "bound": "hbm", "achieved": achieved,
                "peak": hbm, "unit": "GB/s", "frac": achieved / hbm, "traffic": None,
                "algorithmic_bytes_per_launch": bytes_launch,
                "peak_source": "MEASURED_PEAKS.json hbm_gbs (burst copy)" if peaks else "fallback 6.8 TB/s"}
    hbm_src = "MEASURED_PEAKS.json hbm_gbs (burst copy)" if peaks else "fallback 6.8 TB/s"
    roof["family_ms_per_step"] = fam_ms

    if args.profile_run:
        # profiler runs (launch lists, kernel captures): the warm-up and timed steps only
        if rank == 0:
            print(json.dumps({"metric": METRIC, "value": value, "unit": UNIT, "ms_per_step": ms_max / args.steps,
                              "profile_run": True, "roofline": roof, "gpu_launches": launches}))
        P.close()
        return

    # the same steps replayed from the captured CUDA graph (no per-kernel events)
    P.set_graphs(True)
    P.propagate(1)
    torch.cuda.synchronize()
    g0, g1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    n_graph = max(1, min(args.steps, cap - args.warmup - args.steps - 1))
    g0.record(stream)
    P.propagate(n_graph)
    g1.record(stream)
    torch.cuda.synchronize()
    graph_value = n_orb * n_graph * world / (g0.elapsed_time(g1) / 1e3)

    # end-to-end through the C ABI with host buffers: the ground states sit in pinned
    # host memory (filled before the timed region), uploaded inside it
    P.close()
    psi_pinned = torch.from_numpy(psi_host).pin_memory().numpy()
    torch.cuda.synchronize()
    t_e2e = time.perf_counter()
    P2, sids2, _ = build_propagator(args.precision, args.steps, device=local_rank, n_subsims=args.subsims)
    for sid in sids2:
        P2.load_ground_state(sid, psi_pinned)
    P2.set_kick(-1, 0.005, (1.0, 0.0, 0.0))
    P2.propagate(args.steps)
    J_e2e, _ = P2.current(-1)
    torch.cuda.synchronize()
    e2e_s = time.perf_counter() - t_e2e
    P2.close()
    if world > 1:
        e2e_t = torch.tensor([e2e_s], device=f"cuda:{local_rank}")
        dist.all_reduce(e2e_t, op=dist.ReduceOp.MAX)
        e2e_s = float(e2e_t.item())
    e2e = {"value": n_orb * args.steps * world / e2e_s, "unit": UNIT,
           "h2d_bytes_per_step": int(psi_host.nbytes * len(sids2) / args.steps),
           "d2h_bytes_per_step": int(J_e2e.nbytes / max(args.steps, 1)),
           "includes": "context set-up, 64 ground-state uploads (complex128, pinned host memory), kick, "
                       "propagation, two-step current download"}

    # eps(omega) error of this path against the FP64 GPU path (itself pinned to
    # the oracle at err_J <= 1e-10): cell A on its 16^3 grid, MP 2^3, plane-wave
    # start, kick 0.005 x, 600 steps, eps over 0.1-20 eV (Eqs. 12-14)
    eps_err = None
    if args.precision != "fp64":
        eps_err = eps_check(args.precision, local_rank)

    # the enforced-time-reversal-symmetry propagator on the same workload (three
    # Taylor-4 expansions per step: predictor and two half steps)
    etrs = None
    if args.etrs_steps > 0 and args.precision != "fp32_tc":
        P4, sids4, _ = build_propagator(args.precision, args.etrs_steps + 2, device=local_rank,
                                        n_subsims=args.subsims)
        P4.set_propagator("etrs")
        for sid in sids4:
            P4.load_ground_state(sid, psi_dev)
        P4.set_kick(-1, 0.005, (1.0, 0.0, 0.0))
        P4.propagate(1)
        torch.cuda.synchronize()
        s4, e4 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        s4.record(stream)
        P4.propagate(args.etrs_steps)
        e4.record(stream)
        torch.cuda.synchronize()
        etrs_ms = s4.elapsed_time(e4)
        P4.close()
        etrs = {"value": n_orb * args.etrs_steps / (etrs_ms / 1e3), "unit": UNIT, "steps": args.etrs_steps,
                "ms_per_step": etrs_ms / args.etrs_steps,
                "propagator": "ETRS: Taylor-4 predictor for rho(t+dt), then two Taylor-4 half steps"}

    # the per-stage stencil kernel of the dense tensor-core mode, HBM roofline
    stencil = None
    if args.stencil_steps > 0:
        stencil = stencil_roofline(local_rank, args.subsims, hbm, hbm_src, steps=args.stencil_steps)

    # plain FP64 GPU path on the same workload (comparison)
    fp64 = None
    if args.precision != "fp64" and args.fp64_steps > 0:
        P3, sids3, _ = build_propagator("fp64", args.fp64_steps + 1, device=local_rank, n_subsims=args.subsims)
        for sid in sids3:
            P3.load_ground_state(sid, psi_dev)
        P3.set_kick(-1, 0.005, (1.0, 0.0, 0.0))
        P3.propagate(1)
        torch.cuda.synchronize()
        s3, e3 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        s3.record(stream)
        P3.propagate(args.fp64_steps)
        e3.record(stream)
        torch.cuda.synchronize()
        fp64_ms = s3.elapsed_time(e3)
        P3.close()
        fp64 = {"value": n_orb * args.fp64_steps / (fp64_ms / 1e3), "unit": UNIT, "steps": args.fp64_steps,
                "ms_per_step": fp64_ms / args.fp64_steps}

    if rank == 0:
        out = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
               "warmup": args.warmup, "ms_per_step": ms_max / args.steps, "higher_is_better": True,
               "scaling": "weak", "vs_baseline": None, "dtype": "f64" if args.precision == "fp64" else "f32",
               "data": "synthetic (seeded Si-like model, plane-wave start orbitals)",
               "config": {"workload": WORKLOAD if args.subsims == 64 else f"reduced: {args.subsims} of " + WORKLOAD,
                          "n_subsims": len(run.subsims), "k_points": 64 * len(run.subsims),
                          "orbitals_per_gpu": n_orb, "grid": "16^3", "bands": 16, "dt": 0.08,
                          "precision": {"fp32": "fp32 stencil/Taylor; projector contractions factorised per "
                                                "axis, the z contractions as three-product TF32 tensor-core "
                                                "GEMMs (tcgen05, accumulators in tensor memory; mma.sync in "
                                                "variant 3) with fp32 accumulation; fp64 rho/J/Hartree",
                                        "fp32_tc": "fp32 stencil/Taylor; dense projector GEMMs as scaled "
                                                   "split-FP16 three-product tensor-core products (mma.sync) "
                                                   "with fp32 accumulation; fp64 rho/J/Hartree",
                                        "fp64": "fp64 throughout"}[args.precision],
                          "l2": "inputs larger than L2 (psi 2 GiB in fp32), no flush needed",
                          "parallelism": f"shift blocks x{world} (64 independent sub-simulations per GPU, "
                                         "one final all-reduce of dJ)"},
               "roofline": roof, "roofline_stencil": stencil, "e2e": e2e, "gpu_launches": launches,
               "graph_replay_value": graph_value,
               "autotune": {"variant": tuned_variant, "n_variants": tuned_n, "variants_timed": n_tried,
                            "ms_per_step": tuned_ms,
                            "variants": "0 whole step in one launch (z contractions on tcgen05), 1 fused stage "
                                        "per launch (mma.sync), 2 z-march stage with CUDA-core projections, 3 whole "
                                        "step with the z contractions on mma.sync" if tuned_n == 4 else None},
               "clocks": clk.summary(),
               "fp64_gpu": fp64,
               "etrs": etrs,
               "eps_rel_err_vs_fp64": eps_err,
               "eps_check": "cell A (16^3 grid), MP 2^3, plane-wave start, kick 0.005 x, 600 steps, "
                            "eps over 0.1-20 eV vs the FP64 GPU path (FP64 GPU vs oracle: err_J <= 1e-10)",
               "fp32_over_fp64": (value / world / fp64["value"]) if fp64 else None,
               "two_step_dJx_last": float(J_two_step[-1, 0]),
               "two_step_subsims": n_global}
        if cpu is not None:
            out["cpu_baseline"] = cpu
        print(json.dumps(out))
    if world > 1:
        dist.destroy_process_group()


# ----------------------------------------------------------------------------
# Side workloads of the large-cell (point-parallel) path; not the benchmark
# ----------------------------------------------------------------------------
SIDE_WORKLOADS = {
    "cell-b-mp2": "2x2x2 supercell (32^3 grid, 64 atoms, 128 bands), one sub-simulation on a shifted 2^3 "
                  "MP grid (8 k-points), kick 0.005 along x, default kernel variant",
    "uneven": "uneven batch: 18 8-atom 16^3 cells and 2 32^3 supercells with 2^3..6^3 shifted subgrids, "
              "kicks 1e-4..1e-2, autotuned (20 s budget)",
    "config5": "uneven batched two-step run at full size: 180 8-atom 16^3 cells (16 bands) and 20 2x2x2 "
               "supercells (32^3 grid, 64 atoms, 128 bands) with seeded 2^3..6^3 shifted subgrids (19 197 "
               "k-points, 482 208 orbitals), kicks 1e-4..1e-2 along x; plane-wave start orbitals (throughput "
               "only: no ground states for the supercells); default kernel variants (the autotuner's state "
               "snapshot would not fit beside the 185 GB of single-precision state); the seeded 518..4952 step "
               "budgets are capped to the steps run, since the step counts do not change the cost of a step",
    "hhg": "two-step HHG run: 8 shifted 8^3 subgrids of the 8-atom 16^3 cell (4096 k, 65 536 orbitals), the "
           "sin^4 pulse of Eq. 15 along z (E0 0.005, w0 0.057, T 1654), dt 0.04, self-consistent v_Hxc, "
           "plane-wave start; A(t) changes every step, timed from the middle of the pulse",
}


def run_side_workload(args):
    import torch
    import workloads as W
    from paper_2112_00920_gb300 import Propagator, build_library, shifted_kpoints
    build_library()
    cap = args.warmup + args.steps + 40
    P = Propagator(args.precision)
    t_start = 0
    if args.workload == "cell-b-mp2":
        cb = W.cell_b()
        subs = [W.SubsimSpec(cb, (2, 2, 2), (0.5, 0.5, 0.5), 0.08, cap, W.Kick(k0=0.005))]
    elif args.workload == "hhg":
        subs = W.twostep_hhg_run().subsims
        t_start = int(round(0.5 * subs[0].field.t_pulse / subs[0].dt))   # middle of the pulse
    elif args.workload == "config5":
        subs = W.uneven_batch_run(max_steps=cap).subsims
        # device memory: three single-precision orbital arrays (psi and the two
        # Taylor-term buffers) plus projections, partial sums and the largest
        # complex128 upload; refuse rather than run the device out of memory
        orb_bytes = sum(s.mp[0] * s.mp[1] * s.mp[2] * s.cell.n_bands * s.cell.n_pts * 8 for s in subs)
        upload = max(s.mp[0] * s.mp[1] * s.mp[2] * s.cell.n_bands * s.cell.n_pts * 16 for s in subs)
        need = 3 * orb_bytes * 1.08 + 2 * upload
        free, total = torch.cuda.mem_get_info()
        if need > 0.92 * free:
            print(json.dumps({"workload": args.workload, "skipped": f"needs about {need / 1e9:.0f} GB of device "
                              f"memory, {free / 1e9:.0f} GB free"}))
            return
    else:
        subs = W.uneven_batch_run(n_a=18, n_b=2, max_steps=cap).subsims
    cells, sids, n_orb, n_pb = {}, [], 0, 0
    for s in subs:
        if s.cell.name not in cells:
            cells[s.cell.name] = P.add_cell_spec(s.cell)
        sids.append(P.add_subsim(cells[s.cell.name], shifted_kpoints(s.cell.a, s.mp, s.shift), s.dt, cap))
    one_k = {}
    for s, sid in zip(subs, sids):
        c = s.cell
        nk = s.mp[0] * s.mp[1] * s.mp[2]
        if c.name not in one_k:   # the plane-wave start is the same for every k: one set per cell
            one_k[c.name] = torch.from_numpy(W.plane_wave_orbitals(c.a, c.n, W.plane_wave_set(c.n_bands), 1)).cuda()
        psi = one_k[c.name].expand((nk,) + tuple(one_k[c.name].shape[1:])).contiguous()
        P.load_ground_state(sid, psi)
        del psi
        if isinstance(s.field, W.Pulse):
            from paper_2112_00920_gb300 import pulse_samples
            f = s.field
            a = pulse_samples(f.e0, f.omega0, f.t_pulse, f.direction, s.dt, t_start + cap)
            P.set_field(sid, a[2 * t_start:])
        else:
            P.set_kick(sid, s.field.k0, s.field.direction)
        n_orb += nk * c.n_bands
        n_pb += nk * c.n_bands * c.n_pts
    P.propagate(args.warmup)
    tuned = 0
    if args.workload == "uneven":
        tuned = P.autotune(budget_ms=20000)
        P.propagate(1)
    P.set_profiling(True)
    stream = torch.cuda.current_stream()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    l0 = P.launches()
    e0.record(stream)
    P.propagate(args.steps)
    e1.record(stream)
    torch.cuda.synchronize()
    lps = (P.launches() - l0) / args.steps
    ms = e0.elapsed_time(e1) / args.steps
    fam = {k: v / args.steps for k, v in P.timings().items()}
    fam_sum = sum(fam.values())
    out = {"workload": args.workload, "description": SIDE_WORKLOADS[args.workload],
           "n_subsims": len(subs), "orbitals": n_orb,
           "launch_gap_share": (ms - fam_sum) / ms,
           "precision": args.precision, "steps": args.steps, "warmup": args.warmup,
           "ms_per_step": ms, "orbital_steps_per_s": n_orb / (ms / 1e3),
           "point_band_steps_per_s": n_pb / (ms / 1e3), "family_ms_per_step": fam,
           "variants": {name: P.variant(cid) for name, cid in cells.items()},
           "variants_timed": tuned, "launches_per_step": lps}
    if args.workload == "hhg" and args.precision == "fp32":
        v = P.variant(cells[subs[0].cell.name])
        if v[0] in (0, 3) and v[1] == 4:
            peaks = {}
            try:
                peaks = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
            except OSError:
                pass
            out["roofline"] = step_roofline(fam["stage"], n_orb, subs[0].cell, 8, peaks, 0, {},
                                            alu_peaks(torch.cuda.current_device()))
    print(json.dumps(out))
    P.close()


def run_reference(args):
    """The CPU oracle on this host's cores: one process per core, each holding
    one sub-simulation of the benchmark workload; a bench step is one time
    step of all of them (propagate time only)."""
    workers = host_cores()
    pool = OraclePool(workers, args.warmup + args.steps)
    try:
        for _ in range(args.warmup):
            pool.step(1)
        units = 0
        wall = 0.0
        for _ in range(args.steps):
            u, w = pool.step(1)
            units += u
            wall += w
    finally:
        pool.close()
    value = units / wall
    sample = (f"per step: {workers} of the 64 sub-simulations (64 k x 16 bands each) x 1 time step with the "
              f"numpy complex128 oracle, one process per host core, BLAS 1 thread, propagate time only; "
              f"{cpu_model()}")
    out = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
           "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * wall / args.steps,
           "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
           "data": "synthetic (seeded Si-like model, plane-wave start orbitals)",
           "config": {"workload": WORKLOAD, "precision": "fp64 (oracle)"},
           "cpu_baseline": {"value": value, "unit": UNIT, "cores": workers, "kind": "oracle", "sample": sample},
           "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(out))


if __name__ == "__main__":
    main()
