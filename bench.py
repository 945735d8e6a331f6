#!/usr/bin/env python
"""Benchmark: converged one-cell-inversion time steps on one GB300 (or N replicas).

A benchmark step is one time step of the transient problem iterated to the
tolerance (relative change of phi < 1e-8): the whole hot path -- halo gather,
per-ordinate block solves, scattering-moment reduction, capacitance solve,
back-substitution, residual -- every iteration, plus the end-of-step commit.

Default workload: the seeded layered slab (131072 cells in 8-32 layers,
sigma_t = 10^U(-2,2), c ~ U(0, 0.999), optical thickness per cell U(0.05, 5),
sources U(0, 10) on a random half of the layers, S_64, dt = 0.02, v = 1,
vacuum faces, 100-step trajectory from psi0 = 0, tol 1e-8), FP32 angular flux
with compensated moments and double-float capacitance / residual difference.
Its ~212 MB working set exceeds the L2, so every iteration streams from HBM.
``compare`` adds: the 65536-cell homogeneous slab (one point of the quadrature
sweep) as a second headline-style line; the OCI-vs-SI sweep over c, dx and N on
that slab (OCI FP32 / FP64, SI with the paper's march and with the parallel
prefix); SI, FP64 OCI and backward-Euler OCI on the default workload; the error
of the FP32 and BF16-halo paths against the FP64 path per configuration; the
plain-vs-learned-guess comparison on eight thin-cell deployment slabs and one
200-step deployment trajectory; and the dense per-material inverse against the
Woodbury kernel at S_128.  ``value`` = cell-ordinate updates per second (cells
x ordinates x iterations / device time), summed over replicas; ``e2e`` = the
same through the C ABI with pinned host buffers (source in, fluxes out).
Prints one JSON line.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
                  [--workload hetero|slab] [--precision fp32|fp64]
                  [--no-compare] [--no-cpu-baseline]
                  [--only-compare solvers|learned|dense|sweep|errors|deploy200]
"""
import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import workloads  # noqa: E402

METRIC = "cell-ordinate updates/s, OCI to 1e-8 per time step"
UNIT = "cell-ord/s"
TRAFFIC_FILE = os.path.join(ROOT, "profiles", "traffic.txt")
KERNEL_SRC = os.path.join(ROOT, "paper_2305_13555_gb300", "csrc", "oci_device.cuh")


def make_problem(args):
    if args.workload == "slab":
        p = workloads.config2(N=args.n_ord, c=args.c, dx=args.dx, J=args.cells or 65536, n_steps=50)
        desc = (f"homogeneous slab {p['n_cells']} cells, S_{p['n_ord']}, sigma_t=1, c={args.c}, dx={args.dx} mfp, "
                f"dt=0.05, v=1, Q=1, reflect/vacuum, 50-step trajectory, tol 1e-8")
    else:
        p = workloads.config4(seed=args.seed, J=args.cells or 131072, n_steps=100)
        desc = (f"seeded layered slab {p['n_cells']} cells in {int(p['layer'].max()) + 1} layers, S_64, "
                f"sigma_t 10^U(-2,2), c U(0,0.999), tau U(0.05,5), Q U(0,10) on half the layers, dt=0.02, v=1, "
                f"vacuum/vacuum, 100-step trajectory, tol 1e-8 (seed {args.seed})")
    return p, desc


def kernel_hash():
    """Hash of the OCI iteration kernel's source: oci_device.cuh up to the end of the
    staged kernel (everything that kernel can use) and the lines of the FP32
    instantiation file that choose its template arguments."""
    h = hashlib.sha256()
    text = open(KERNEL_SRC, "rb").read()
    cut = text.find(b"// Per-cell passes without reductions")
    h.update(text if cut < 0 else text[:cut])
    for line in open(os.path.join(ROOT, "paper_2305_13555_gb300", "csrc", "oci_kernels_f32.cu"), "rb"):
        if b"kStages" in line or b"k_cells_tma" in line or b"fill<" in line:
            h.update(line)
    return h.hexdigest()[:16]


def read_traffic(key):
    """Per-launch DRAM bytes of the iteration kernel from the committed ncu
    summary, if it was taken on the current kernel source."""
    if not os.path.exists(TRAFFIC_FILE):
        return None
    for line in open(TRAFFIC_FILE):
        parts = line.split()
        if len(parts) >= 3 and not line.startswith("#") and parts[0] == key and parts[1] == kernel_hash():
            return float(parts[2])
    return None


NOMINAL_HBM_GBS = 7900.0  # GB300 HBM3e, nominal (the measured copy bandwidth is the roofline's peak)


def load_peaks():
    try:
        return json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json"))), "measured"
    except Exception:
        return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0}, "fallback"


class ClockSampler:
    """nvidia-smi clocks / throttle reasons every 100 ms, each line stamped on
    arrival; only the lines stamped inside the timed region count."""
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.gpu = gpu_index
        self.proc = None
        self.lines = []
        self.reader = None

    def start(self):
        """Starts nvidia-smi and returns once its first line has arrived (or after 3 s)."""
        import threading
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.Q}",
                                          "--format=csv,noheader,nounits", "-lms", "10"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except Exception:
            self.proc = None
            return

        def read():
            for line in self.proc.stdout:
                self.lines.append((time.perf_counter(), line))

        self.reader = threading.Thread(target=read, daemon=True)
        self.reader.start()
        t_end = time.perf_counter() + 3.0
        while not self.lines and time.perf_counter() < t_end:
            time.sleep(0.01)

    def stop(self, t0, t1):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
            self.proc.wait()
        self.reader.join(timeout=5)
        return self.summarize(self.lines, t0, t1)

    @staticmethod
    def summarize(lines, t0, t1, margin=0.25):
        """Median SM clock, maximum clock and active slowdown reasons of the
        (arrival time, csv line) samples stamped inside [t0, t1].  A timed
        region shorter than the sampling period may hold no sample: then the
        samples within `margin` seconds on either side stand in, marked
        "adjacent"."""
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        parsed = []
        for t, line in lines:
            f = [x.strip() for x in line.split(",")]
            if len(f) < 9:
                continue
            try:
                sm, smax = float(f[1]), float(f[2])
            except ValueError:
                continue
            parsed.append((t, sm, smax, {n for n, v in zip(names, f[5:9]) if v.lower() == "active"}))
        inside = [s for s in parsed if t0 <= s[0] <= t1]
        adjacent = False
        if not inside:
            inside = [s for s in parsed if t0 - margin <= s[0] <= t1 + margin]
            adjacent = bool(inside)
        if not inside:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": [], "samples": 0,
                    "note": "no clock sample inside or next to the timed region"}
        out = {"sm_mhz": statistics.median(s[1] for s in inside), "sm_max_mhz": max(s[2] for s in inside),
               "reasons": sorted(set().union(*(s[3] for s in inside))), "samples": len(inside),
               "timed_region_s": round(t1 - t0, 3)}
        if adjacent:
            out["adjacent"] = True
            out["note"] = f"timed region shorter than the sampling period: samples within {margin} s of it"
        return out


def aggregate(dev_time, units, device="cpu"):
    """Replicas: the job's time is the slowest rank's, its work the sum over ranks."""
    import torch
    t = torch.tensor([dev_time, units], dtype=torch.float64, device=device)
    tmax = t.clone()
    torch.distributed.all_reduce(tmax, op=torch.distributed.ReduceOp.MAX)
    torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.SUM)
    return float(tmax[0]), float(t[1])


def trajectory_chunks(k0, steps, n_traj, ch):
    """Calls of the end-to-end leg: (restart from psi0 before the call, steps in
    the call) for `steps` more steps of a trajectory of n_traj steps replayed
    from psi0, k0 steps already run; a call never runs across a restart and has
    at most ch steps."""
    out, k, done = [], k0, 0
    while done < steps:
        m = min(ch, steps - done, n_traj - k % n_traj)
        out.append((k > 0 and k % n_traj == 0, m))
        k += m
        done += m
    return out


def algorithmic_bytes(J, N, rs):
    """Bytes one OCI iteration must move: per cell-ordinate 2 incident values,
    2 time-edge values, 2 outgoing values (6 words); per cell phi^l in and
    phi^{l+1} out (8 doubles), the source moments (4 words) and a material id."""
    return 6 * J * N * rs + J * (64 + 4 * rs + 4)


def run_ours(args, rank, world):
    import torch
    import paper_2305_13555_gb300 as pkg

    dev = int(os.environ.get("LOCAL_RANK", 0))
    torch.cuda.set_device(dev)
    pkg.load_library()
    prob, desc = make_problem(args)
    J, N = prob["n_cells"], prob["n_ord"]
    rs = 4 if args.precision == "fp32" else 8
    stream = torch.cuda.current_stream()
    flush = torch.empty(256 << 20, dtype=torch.uint8, device="cuda")
    s = pkg.Solver(prob, precision=args.precision, tol=prob["tol"], stream=stream.cuda_stream)
    # the workload is a trajectory of n_steps time steps from psi0 = 0; longer runs
    # replay it, restarting from the initial condition through oci_set_state
    n_traj = prob["n_steps"]
    psi_init = torch.zeros((J, N, 2), dtype=torch.float64).pin_memory().numpy()
    counter = {"k": 0, "restarts": 0}

    def restart_if_due():
        """Returns the library kernels the restart launched (one conversion kernel)."""
        due = counter["k"] and counter["k"] % n_traj == 0
        if due:
            s.set_state(psi_init)
            counter["restarts"] += 1
        counter["k"] += 1
        return 1 if due else 0

    for _ in range(args.warmup):
        restart_if_due()
        rc, st = s.step()
        assert rc == pkg.OCI_OK, (rc, st)
    if world > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    clocks = ClockSampler(dev)
    clocks.start()
    iters, secs, launches = [], [], 0
    t_wall0 = time.perf_counter()
    for _ in range(args.steps):
        launches += restart_if_due()  # host call between steps, outside the steps' device time
        flush.zero_()  # evict the previous step's data from L2 between timed steps
        rc, st = s.step()
        assert rc == pkg.OCI_OK, (rc, st)
        iters.append(st["iters"])
        secs.append(st["seconds"])
        launches += st["launches"]  # kernels of the library for the step (as counted by oci_step)
    torch.cuda.synchronize()
    wall = time.perf_counter() - t_wall0
    clk = clocks.stop(t_wall0, t_wall0 + wall)
    dev_time = float(sum(secs))
    units = float(J) * N * float(sum(iters))
    if world > 1:
        dev_time, units = aggregate(dev_time, units, "cuda")
    value = units / dev_time

    # roofline: the iteration alone, CUDA events on the same stream (the FP32 path
    # runs the 50 iterations as one persistent cooperative launch)
    t_launch = pkg.oci_profile_iterations(s.h, 50)
    abytes = algorithmic_bytes(J, N, rs)
    peaks, peak_kind = load_peaks()
    peak = float(peaks["hbm_gbs"])
    achieved = abytes / t_launch / 1e9
    traffic = read_traffic(f"{args.workload}_{args.precision}_S{N}_J{J}")
    roofline = {"bound": "hbm", "achieved": round(achieved, 1), "peak": peak, "unit": "GB/s",
                "frac": round(achieved / peak, 4), "traffic": traffic, "peak_source": peak_kind,
                "nominal_peak_gbs": NOMINAL_HBM_GBS, "frac_of_nominal": round(achieved / NOMINAL_HBM_GBS, 4),
                "kernel": ("k_cells_tma<OCI> persistent loop (figures per iteration; 50 iterations per launch)"
                           if args.precision == "fp32" else "k_cells<double, OCI> (one launch per iteration)"),
                "iteration_us": round(t_launch * 1e6, 3), "algorithmic_bytes_per_iteration": abytes,
                "algorithmic_bytes": "24 B per cell-ordinate (2 incident, 2 time-edge, 2 outgoing words) + 84 B per "
                                     "cell (phi in and out as double-float, source moments, material id)"
                                     if rs == 4 else "48 B per cell-ordinate + 100 B per cell",
                "working_set_vs_l2": f"{abytes / 1e6:.0f} MB per iteration against a 129 MB L2"}

    # end to end through the C ABI with host buffers: each step's source in and
    # its fluxes out, in pinned host memory (page-locked, so the copies are
    # direct DMA), through oci_run_steps: the next step is queued on the device
    # before the host waits for the current one, the copies run on the library's
    # copy streams; calls of at most 32 steps, the trajectory restarts between them
    CH = 32
    q_pin = torch.empty((CH, J, 4), dtype=torch.float64).pin_memory()
    phi_pin = torch.empty((CH, J, 4), dtype=torch.float64).pin_memory()
    q_host, phi_host = q_pin.numpy(), phi_pin.numpy()
    q_host[:] = np.asarray(prob["q"], dtype=np.float64).reshape(1, J, 4)
    e2e_iters = 0
    r0 = counter["restarts"]
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for restart, m in trajectory_chunks(counter["k"], args.steps, n_traj, CH):
        if restart:
            s.set_state(psi_init)
            counter["restarts"] += 1
        counter["k"] += m
        rc, done, stats = pkg.oci_run_steps(s.h, m, q_host[:m], phi_host[:m])
        assert rc == pkg.OCI_OK and done == m, (rc, done, stats)
        e2e_iters += sum(st["iters"] for st in stats)
    e2e_t = time.perf_counter() - t0
    state_bytes = (counter["restarts"] - r0) * psi_init.nbytes  # initial conditions of the replayed trajectories
    e2e = {"value": float(J) * N * e2e_iters / e2e_t, "unit": UNIT,
           "h2d_bytes_per_step": int(q_host[0].nbytes + state_bytes / args.steps),
           "d2h_bytes_per_step": int(phi_host[0].nbytes),
           "h2d": "source Q each step, initial angular flux psi0 at each trajectory restart (pinned host memory)",
           "api": "oci_run_steps: two steps in flight, sources up and moments down on the library's upload and copy streams"}
    s.close()

    compare = {}
    if not args.no_compare and rank == 0:
        compare = run_compare(args, pkg, torch, stream)
        compare["slab_65536"] = run_slab_point(args, pkg, torch, stream)
        compare["err_vs_fp64"] = run_errors(args, pkg, torch, stream)
        compare["sweep_oci_vs_si"] = run_sweep(args, pkg, torch, stream)
        compare["learned_guess"] = run_learned(args, pkg, torch, stream)
        compare["deploy_200_steps"] = run_deploy200(args, pkg, torch, stream)
        compare["dense_inverse_s128"] = run_dense(args, pkg, torch, stream)
    return {
        "n_traj": n_traj, "value": value, "units": units, "dev_time": dev_time, "wall": wall, "iters": iters, "launches": launches,
        "roofline": roofline, "e2e": e2e, "clocks": clk, "desc": desc, "J": J, "N": N, "compare": compare,
    }


def run_compare(args, pkg, torch, stream):
    """SI (the paper's sequential sweep, and the parallel-prefix sweep), FP64 OCI,
    the backward-Euler time scheme, FP32 OCI started from the extrapolation in
    time and the BF16 halo on the same problem (fewer steps), for context."""
    out = {}
    prob, _ = make_problem(args)
    J, N = prob["n_cells"], prob["n_ord"]
    for name, method, prec, sweep, scheme, halo in (
            ("si_" + args.precision, "si", args.precision, "march", "mb", "fp32"),
            ("si_scan_" + args.precision, "si", args.precision, "scan", "mb", "fp32"),
            ("oci_fp64", "oci", "fp64", "march", "mb", "fp32"),
            ("si_fp64", "si", "fp64", "march", "mb", "fp32"),
            ("si_scan_fp64", "si", "fp64", "scan", "mb", "fp32"),
            ("oci_backward_euler_fp32", "oci", "fp32", "march", "be", "fp32"),
            ("oci_backward_euler_fp64", "oci", "fp64", "march", "be", "fp32"),
            ("oci_fp32_same_window", "oci", "fp32", "march", "mb", "fp32"),
            ("oci_fp32_extrapolated", "oci", "fp32", "march", "mb", "fp32"),
            ("oci_fp32_bf16_halo", "oci", "fp32", "march", "mb", "bf16")):
        if (halo == "bf16" or name.startswith("oci_fp32_")) and args.precision != "fp32":
            continue
        s = pkg.Solver(prob, precision=prec, tol=prob["tol"], stream=stream.cuda_stream, sweep=sweep, scheme=scheme,
                       halo=halo, guess="extrapolate" if name == "oci_fp32_extrapolated" else "previous")
        n_w, n_t = 2, min(args.steps, 5)
        its, secs = [], []
        ok = True
        for k in range(n_w + n_t):
            rc, st = s.step(method)
            if rc != pkg.OCI_OK:
                ok = False
                break
            if k >= n_w:
                its.append(st["iters"])
                secs.append(st["seconds"])
        t_it = pkg.oci_profile_iterations(s.h, 20) if (ok and method == "oci") else None
        s.close()
        if ok:
            out[name] = {"updates_per_s": J * N * sum(its) / sum(secs), "s_per_step": sum(secs) / len(secs),
                         "iters_per_step": sum(its) / len(its)}
            if t_it is not None:
                out[name]["s_per_iteration"] = t_it
    return out


def _run_steps(pkg, stream, prob, n_steps, precision="fp32", method="oci", sweep="march", halo="fp32", tol=None,
               nn=0, W=None, k_corr=50, max_iter=100000, keep_phi=False, skip=0, cap=None, guess="previous"):
    """Steps 1..n_steps of a trajectory from psi0 on one handle: per-step device
    seconds and iterations (steps after the first ``skip`` are summarised), the
    published fluxes of every step if asked, or the failing status.  With
    ``cap``, a step stops after that many iterations and is committed anyway;
    such steps are counted (the FP32 sweeps can stall at the rounding floor just
    above the tolerance)."""
    tol = prob["tol"] if tol is None else tol
    s = pkg.Solver(prob, precision=precision, tol=tol, stream=stream.cuda_stream, max_iter=max_iter, sweep=sweep,
                   halo=halo, guess=guess)
    capped, worst = 0, 0.0
    try:
        if nn:
            pkg.oci_nn_attach(s.h, W, nn, k_corr)
        if cap:
            s.set_iteration(tol, cap, commit_unconverged=True)
        its, secs, phis = [], [], []
        for k in range(n_steps):
            rc, st = s.step(method)
            if cap and rc == pkg.OCI_ENOTCONV and st["committed"]:
                capped += 1
                worst = max(worst, st["residual"])
            elif rc != pkg.OCI_OK:
                return {"failed_status": rc, "failed_at_step": k + 1}
            its.append(st["iters"])
            secs.append(st["seconds"])
            if keep_phi:
                phis.append(s.fluxes())
    finally:
        s.close()
    J, N = prob["n_cells"], prob["n_ord"]
    ti, ts = its[skip:], secs[skip:]
    out = {"s_per_step": sum(ts) / len(ts), "iters_per_step": sum(ti) / len(ti),
           "updates_per_s": J * N * sum(ti) / sum(ts), "steps": f"{skip + 1}-{n_steps}"}
    if cap:
        out.update(steps_at_cap=capped, worst_residual_at_cap=worst)
    if keep_phi:
        out["phi"] = phis
    return out


def run_slab_point(args, pkg, torch, stream):
    """The 65536-cell homogeneous slab (S_64, c = 0.9, dx = 0.1 mfp, reflecting
    left / vacuum right, dt = 0.05): its 50-step trajectory and the iteration
    kernel's roofline there (working set ~106 MB, inside the L2 across the
    iterations of a step, so that fraction is not an HBM figure)."""
    prob = workloads.config2(N=64, c=0.9, dx=0.1, J=65536, n_steps=50)
    rec = _run_steps(pkg, stream, prob, 50)
    s = pkg.Solver(prob, precision="fp32", tol=prob["tol"], stream=stream.cuda_stream)
    t = pkg.oci_profile_iterations(s.h, 50)
    s.close()
    peak = float(load_peaks()[0]["hbm_gbs"])
    b = algorithmic_bytes(65536, 64, 4)
    rec.update(workload="homogeneous slab 65536 cells, S_64, c=0.9, dx=0.1 mfp, dt=0.05, reflect/vacuum, 50 steps",
               iteration_us=round(t * 1e6, 3), achieved_gbs=round(b / t / 1e9, 1),
               frac_l2_assisted=round(b / t / 1e9 / peak, 4), traffic=read_traffic("slab_fp32_S64_J65536"),
               note="working set ~106 MB stays in L2 across a step's iterations: algorithmic bytes over the HBM "
                    "copy peak, not an HBM fraction")
    return rec


def _maxrel(a, b):
    return float(np.abs(np.asarray(a) - np.asarray(b)).max() / max(np.abs(np.asarray(b)).max(), 1e-300))


def run_errors(args, pkg, torch, stream):
    """Error of the reduced-precision paths against the FP64 path per
    configuration: the published scalar-flux moments of every step of a
    trajectory, FP32 (and the BF16 incident-flux halo) at the configuration's
    tolerance against FP64 OCI converged to 1e-12 (the FP64 path matches the FP64
    oracle to 1e-12 at a fixed iteration count); max over the steps of
    max|phi - phi_ref| / max|phi_ref|.  FP64 at the configuration's tolerance is
    listed too: what of the error is the stopping tolerance, not the rounding."""
    cases = [
        ("config2_slab65536_S64_c0.9_dx0.1", workloads.config2(N=64, c=0.9, dx=0.1, J=65536, n_steps=50), 50),
        ("config3_slab16384_S128", workloads.config3(n_steps=20), 20),
        (f"config4_layered131072_S64_seed{args.seed}", workloads.config4(seed=args.seed, n_steps=100), 100),
        (f"config5_deploy131072_S64_seed{args.nn_seed}", workloads.config5_deploy(args.nn_seed, n_steps=10), 10),
    ]
    out = {"definition": "max over steps of max|phi - phi_fp64| / max|phi_fp64| (4 moments, all cells); "
                         "reference: GPU FP64 OCI at tol 1e-12"}
    for name, prob, n in cases:
        ref = _run_steps(pkg, stream, prob, n, "fp64", tol=1e-12, keep_phi=True)
        if "phi" not in ref:
            out[name] = {"reference_failed": ref}
            continue
        rec = {"steps": n, "tol": prob["tol"]}
        for key, prec, halo in (("fp32", "fp32", "fp32"), ("fp32_bf16_halo", "fp32", "bf16"), ("fp64", "fp64", "fp32")):
            if halo == "bf16" and prob["n_ord"] % 8:
                continue
            r = _run_steps(pkg, stream, prob, n, prec, halo=halo, keep_phi=True)
            rec[key] = (max(_maxrel(a, b) for a, b in zip(r["phi"], ref["phi"])) if "phi" in r else r)
        out[name] = rec
    return out


def run_sweep(args, pkg, torch, stream, n_steps=None):
    """OCI against SI on the 65536-cell homogeneous slab over the scattering
    ratio, the cell width and the quadrature order (c in {0.5, 0.9, 0.99}, dx in
    {0.01, 0.1, 1, 10} mfp, S_32 and S_64; Sigma = 1, dt = 0.05, reflecting left /
    vacuum right, tol 1e-8): iterations and device seconds per converged step
    over the trajectory's first steps, for OCI in FP32 and FP64, FP32 OCI started
    from the extrapolation in time, SI with the paper's march and SI with the
    parallel prefix (FP32), the latter also from the extrapolated start."""
    n_steps = n_steps or args.sweep_steps
    rows = []
    for N in (32, 64):
        for c in (0.5, 0.9, 0.99):
            for dx in (0.01, 0.1, 1.0, 10.0):
                prob = workloads.config2(N=N, c=c, dx=dx, J=65536, n_steps=n_steps)
                row = {"N": N, "c": c, "dx": dx}
                for key, prec, method, sweep, guess in (
                        ("oci_fp32", "fp32", "oci", "march", "previous"), ("oci_fp64", "fp64", "oci", "march", "previous"),
                        ("oci_fp32_extrapolated", "fp32", "oci", "march", "extrapolate"),
                        ("si_march_fp32", "fp32", "si", "march", "previous"),
                        ("si_scan_fp32", "fp32", "si", "scan", "previous"),
                        ("si_scan_fp32_extrapolated", "fp32", "si", "scan", "extrapolate")):
                    r = _run_steps(pkg, stream, prob, n_steps, prec, method, sweep, cap=500, guess=guess)
                    row[key] = ({"iters": round(r["iters_per_step"], 2), "ms": round(r["s_per_step"] * 1e3, 4)}
                                if "s_per_step" in r else r)
                    if r.get("steps_at_cap"):
                        row[key].update(steps_at_cap=r["steps_at_cap"], worst_residual=r["worst_residual_at_cap"])
                # best SI: the faster of the two sweeps among those whose every step reached the tolerance
                best_si = min((row[k]["ms"] for k in ("si_march_fp32", "si_scan_fp32")
                               if "ms" in row[k] and not row[k].get("steps_at_cap")), default=None)
                if "ms" in row["oci_fp32"] and "ms" in row["si_march_fp32"] and not row["si_march_fp32"].get("steps_at_cap"):
                    row["si_march_over_oci_fp32_time"] = round(row["si_march_fp32"]["ms"] / row["oci_fp32"]["ms"], 3)
                if "ms" in row["oci_fp32"] and best_si is not None:
                    row["best_si_over_oci_fp32_time"] = round(best_si / row["oci_fp32"]["ms"], 3)
                if "ms" in row["oci_fp32_extrapolated"] and best_si is not None:
                    row["best_si_over_oci_fp32_extrapolated_time"] = round(best_si / row["oci_fp32_extrapolated"]["ms"], 3)
                se, oe = row["si_scan_fp32_extrapolated"], row["oci_fp32_extrapolated"]
                if "ms" in se and "ms" in oe and not se.get("steps_at_cap"):  # like for like: both extrapolated
                    row["si_scan_over_oci_fp32_both_extrapolated_time"] = round(se["ms"] / oe["ms"], 3)
                rows.append(row)
    return {"workload": f"homogeneous slab 65536 cells, Sigma=1, dt=0.05, v=1, Q=1, reflect/vacuum, tol 1e-8; "
                        f"steps 1-{n_steps} of each trajectory from psi0 = 0",
            "paper_context": "paper: up to 3.4x OCI over SI wall clock (RTX 2060 mobile, CuPy/cuSPARSE GMRES, "
                             "homogeneous slab L=10, Sigma=2, Q=0.1, 5 steps); context only",
            "rows": rows}


# Deployment slabs on which the learned guess is evaluated, fixed before any was
# measured (the four slabs looked at while the method was built, 7-10, are not
# among them).
GAIN_SEEDS = (101, 102, 103, 104, 105, 106, 107, 108)


def run_learned(args, pkg, torch, stream):
    """The metric's "plain vs NN+FP32" part on thin-cell deployment slabs
    (131072 cells, S_64, sigma_t dx ~ U(0.01, 0.1), c ~ U(0.9, 0.999), dt = 0.02):
    seconds and iterations per converged step of plain FP32 OCI and FP32 OCI with
    the trained network (the guess on every step, and the adaptive mode that keeps
    it only where a plain/guessed trial shows a gain) on eight seeded slabs fixed
    in advance, steps 3-8 of each trajectory (2 steps in, the same initial state)."""
    from paper_2305_13555_gb300 import learned
    if not os.path.exists(learned.DEFAULT_WEIGHTS):
        return {"unavailable": "no trained weights"}
    W = learned.load_weights()
    out = {"workload": "config-5 deployment slabs: 131072 cells, S_64, thin cells (sigma_t dx 0.01-0.1), "
                       "c 0.9-0.999, dt 0.02, vacuum/vacuum, tol 1e-8; steps 3-8", "seeds": list(GAIN_SEEDS)}
    per_seed = {}
    for seed in GAIN_SEEDS:
        prob = workloads.config5_deploy(seed, J=131072, N=64, n_steps=8)
        rec = {}
        for key, nn, guess in (("fp32_plain", 0, "previous"), ("fp32_nn_guess", pkg.OCI_NN_GUESS, "previous"),
                               ("fp32_nn_adaptive", pkg.OCI_NN_GUESS_ADAPTIVE, "previous"),
                               ("fp32_extrapolated", 0, "extrapolate"),
                               ("fp32_extrapolated_nn_adaptive", pkg.OCI_NN_GUESS_ADAPTIVE, "extrapolate")):
            r = _run_steps(pkg, stream, prob, 8, "fp32", nn=nn, W=W, max_iter=50000, skip=2, guess=guess)
            rec[key] = r
        per_seed[str(seed)] = rec
    out["per_seed"] = per_seed
    out["inference_breakdown_us"] = nn_breakdown(pkg, torch, W, stream)
    for key in ("fp32_nn_guess", "fp32_nn_adaptive", "fp32_extrapolated", "fp32_extrapolated_nn_adaptive"):
        ok = [r for r in per_seed.values() if "s_per_step" in r["fp32_plain"] and "s_per_step" in r[key]]
        if ok:
            out[f"{key}_over_plain_time_ratio_mean"] = sum(r[key]["s_per_step"] / r["fp32_plain"]["s_per_step"]
                                                           for r in ok) / len(ok)
            out[f"{key}_over_plain_iters_ratio_mean"] = sum(r[key]["iters_per_step"] / r["fp32_plain"]["iters_per_step"]
                                                            for r in ok) / len(ok)
    return out


def nn_breakdown(pkg, torch, W, stream, J=131072, reps=50):
    """Device time of the network's parts for one 131072-cell sample of the
    first deployment slab (learned.time_inference: CUDA events on the launching
    stream, mean of reps after warm-up)."""
    from paper_2305_13555_gb300 import learned
    prob = workloads.config5_deploy(GAIN_SEEDS[0], J=J, N=64, n_steps=2)
    s = pkg.Solver(prob, precision="fp32", tol=1e-8, stream=stream.cuda_stream)
    stat = torch.empty((1, J, 4), dtype=torch.float32, device="cuda")
    qf = torch.empty((1, J), dtype=torch.float32, device="cuda")
    pkg.oci_nn_static_features(s.h, stat, qf)
    s.close()
    return learned.time_inference(W, J, reps=reps, stat=stat, qfeat=qf, stream=stream)


def run_deploy200(args, pkg, torch, stream):
    """One whole 200-step deployment trajectory (131072 cells, S_64, thin cells,
    c 0.9-0.999, dt 0.02, tol 1e-8, seed --nn-seed): device seconds and
    iterations per converged step of plain FP32 OCI (from the previous step's
    flux, and from its extrapolation in time), FP32 OCI with the learned guess
    (adaptive, always, adaptive on the extrapolated start), plain FP64 OCI, and
    SI (FP32, the paper's march and the parallel prefix, the latter also from
    the extrapolated start)."""
    from paper_2305_13555_gb300 import learned
    W = learned.load_weights() if os.path.exists(learned.DEFAULT_WEIGHTS) else None
    n = args.deploy_steps
    prob = workloads.config5_deploy(args.nn_seed, J=131072, N=64, n_steps=n)
    out = {"workload": f"deployment slab 131072 cells, S_64, seed {args.nn_seed}, steps 1-{n}, tol 1e-8"}
    P, E = "previous", "extrapolate"
    runs = [("oci_fp32_plain", "fp32", "oci", "march", 0, P), ("oci_fp32_extrapolated", "fp32", "oci", "march", 0, E),
            ("oci_fp64_plain", "fp64", "oci", "march", 0, P),
            ("si_march_fp32", "fp32", "si", "march", 0, P), ("si_scan_fp32", "fp32", "si", "scan", 0, P),
            ("si_scan_fp32_extrapolated", "fp32", "si", "scan", 0, E), ("si_scan_fp64", "fp64", "si", "scan", 0, P)]
    if W is not None:
        runs.insert(2, ("oci_fp32_nn_adaptive", "fp32", "oci", "march", pkg.OCI_NN_GUESS_ADAPTIVE, P))
        runs.insert(3, ("oci_fp32_nn_guess", "fp32", "oci", "march", pkg.OCI_NN_GUESS, P))
        runs.insert(4, ("oci_fp32_extrapolated_nn_adaptive", "fp32", "oci", "march", pkg.OCI_NN_GUESS_ADAPTIVE, E))
    for key, prec, method, sweep, nn, guess in runs:
        out[key] = _run_steps(pkg, stream, prob, n, prec, method, sweep, nn=nn, W=W, max_iter=50000, guess=guess)
    return out


def run_dense(args, pkg, torch, stream):
    """The dense per-material inverse variant against the Woodbury kernels on
    the S_128 slab (16384 cells, c = 0.9, dx = 1 mfp; 512 x 512 inverse):
    device seconds per iteration (CUDA events, 20 iterations) and per converged
    step, FP64 and FP32.  The dense iteration's GEMM does 2 (4N)^2 flop per
    cell; its rate is reported in TFLOP/s."""
    prob = workloads.config3(n_steps=4)
    J, N = prob["n_cells"], prob["n_ord"]
    out = {"workload": "slab 16384 cells, S_128, sigma_t=1, c=0.9, dx=1 mfp, dt=0.05, reflect/vacuum, tol 1e-8"}
    for prec in ("fp64", "fp32"):
        for solver in ("woodbury", "dense"):
            s = pkg.Solver(prob, precision=prec, tol=prob["tol"], stream=stream.cuda_stream, solver=solver)
            rec = {}
            if prec == "fp64":
                its, secs = [], []
                for k in range(3):
                    rc, st = s.step()
                    if rc != pkg.OCI_OK:
                        rec["failed_status"] = rc
                        break
                    if k >= 1:
                        its.append(st["iters"])
                        secs.append(st["seconds"])
                if its:
                    rec.update(s_per_step=sum(secs) / len(secs), iters_per_step=sum(its) / len(its))
            t = pkg.oci_profile_iterations(s.h, 20)
            rec["s_per_iteration"] = t
            rec["updates_per_s"] = J * N / t
            if solver == "dense":
                rec["gemm_tflops_incl_rhs_out"] = 2.0 * (4 * N) ** 2 * J / t / 1e12
            s.close()
            out[f"{solver}_{prec}"] = rec
    return out


def cpu_baseline(args, seconds_target=15.0):
    """The FP64 oracle (dense LU per cell) on the host cores: OCI iterations of
    the same problem, as many as fit about seconds_target."""
    import oracle
    prob, _ = make_problem(args)
    J, N = prob["n_cells"], prob["n_ord"]
    P = oracle.Problem(prob)
    t0 = time.perf_counter()
    oracle.run(P, "oci", 1, tol=0.0, max_iter=1, commit_unconverged=True)
    t1 = time.perf_counter() - t0
    m = int(max(1, min(50, seconds_target / max(t1, 1e-3))))
    t0 = time.perf_counter()
    oracle.run(P, "oci", 1, tol=0.0, max_iter=m, commit_unconverged=True)
    t = time.perf_counter() - t0
    return {"value": J * N * m / t, "unit": UNIT, "cores": oracle.max_threads(), "kind": "oracle",
            "sample": f"{m} OCI iterations (FP64 dense LU per cell) of one time step of the same {J}-cell S_{N} "
                      f"problem, {t:.1f} s"}


def run_reference(args, budget_s=150.0):
    """The oracle as the reference arm: each step a bounded sample of the
    workload timed on the host cores, sized so that warm-up plus timed steps
    take about budget_s: two OCI iterations of the whole problem per step when
    they fit, else one iteration of a slab of the same recipe with fewer cells."""
    import oracle
    prob, desc = make_problem(args)
    J, N = prob["n_cells"], prob["n_ord"]
    P = oracle.Problem(prob)
    t0 = time.perf_counter()
    oracle.run(P, "oci", 1, tol=0.0, max_iter=1, commit_unconverged=True)
    t_iter = time.perf_counter() - t0
    per_step_budget = budget_s / max(1, args.steps + args.warmup)
    per_step, Js = 2, J
    if 2 * t_iter > per_step_budget:
        per_step = 1
        if t_iter > per_step_budget:
            Js = max(1024, int(J * per_step_budget / t_iter) // 256 * 256)
            sub = argparse.Namespace(**vars(args))
            sub.cells = Js
            P = oracle.Problem(make_problem(sub)[0])
    for _ in range(args.warmup):
        oracle.run(P, "oci", 1, tol=0.0, max_iter=1, commit_unconverged=True)
    its, secs = 0, 0.0
    for _ in range(args.steps):
        t0 = time.perf_counter()
        oracle.run(P, "oci", 1, tol=0.0, max_iter=per_step, commit_unconverged=True)
        secs += time.perf_counter() - t0
        its += per_step
    value = Js * N * its / secs
    sample = f"{per_step} OCI iteration(s) per step of the {J}-cell S_{N} problem"
    if Js != J:
        sample = f"1 OCI iteration per step of a {Js}-cell slab of the same recipe (the {J}-cell S_{N} problem scaled down)"
    return {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": secs / args.steps * 1e3,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": desc, "parallelism": "host threads (OpenMP)"},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": oracle.max_threads(), "kind": "oracle",
                         "sample": sample},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=1000)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="hetero", choices=["hetero", "slab"])
    ap.add_argument("--precision", default="fp32", choices=["fp32", "fp64"])
    ap.add_argument("--n-ord", type=int, default=64)
    ap.add_argument("--cells", type=int, default=0, help="0: the workload's own size")
    ap.add_argument("--c", type=float, default=0.9)
    ap.add_argument("--dx", type=float, default=0.1)
    ap.add_argument("--seed", type=int, default=4)
    ap.add_argument("--nn-seed", type=int, default=GAIN_SEEDS[0])
    ap.add_argument("--no-compare", action="store_true")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--sweep-steps", type=int, default=50)
    ap.add_argument("--deploy-steps", type=int, default=200)
    ap.add_argument("--only-compare", choices=["solvers", "learned", "dense", "sweep", "errors", "deploy200", "slab"],
                    help="run one comparison block alone and print it (for profiling its kernels)")
    args = ap.parse_args()
    args.warmup = max(args.warmup, 3)

    if args.only_compare:
        import torch
        import paper_2305_13555_gb300 as pkg
        pkg.load_library()
        stream = torch.cuda.current_stream()
        fn = {"solvers": run_compare, "learned": run_learned, "dense": run_dense, "sweep": run_sweep,
              "errors": run_errors, "deploy200": run_deploy200, "slab": run_slab_point}[args.only_compare]
        print(json.dumps({args.only_compare: fn(args, pkg, torch, stream)}))
        return

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))

    if args.impl == "reference":
        if rank == 0:
            print(json.dumps(run_reference(args)))
        return

    if world > 1:
        import torch
        torch.distributed.init_process_group("nccl")
    r = run_ours(args, rank, world)
    if rank == 0:
        cpu = None if args.no_cpu_baseline or world > 1 else cpu_baseline(args)
        out = {
            "metric": METRIC, "value": r["value"], "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": r["dev_time"] / args.steps * 1e3, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32" if args.precision == "fp32" else "f64",
            "data": "synthetic",
            "config": {"workload": r["desc"], "cells": r["J"], "ordinates": r["N"],
                       "parallelism": "replicas" if world > 1 else "single GPU",
                       "l2": "flushed (256 MiB write) between timed steps; the working set (~212 MB per iteration "
                             "at 131072 cells, S_64) exceeds the 129 MB L2" if r["J"] * r["N"] * 24 > 129e6 else
                             "flushed (256 MiB write) between timed steps; iterations within a step reuse L2",
                       "trajectory": f"{r['n_traj']} time steps from psi0 = 0, replayed from psi0 (oci_set_state) "
                                     f"when warm-up + timed steps exceed it"},
            "iters_per_step": sum(r["iters"]) / len(r["iters"]),
            "s_per_step": r["dev_time"] / args.steps,
            "roofline": r["roofline"], "cpu_baseline": cpu, "e2e": r["e2e"], "gpu_launches": r["launches"],
            "clocks": r["clocks"], "compare": r["compare"],
        }
        print(json.dumps(out))
    if world > 1:
        import torch
        torch.distributed.destroy_process_group()


if __name__ == "__main__":
    main()
