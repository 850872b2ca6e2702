"""Benchmark of the immersed Newmark IMEX time step on GB300.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl gb300|reference]

One bench "step" is one IMEX time step (Fig. TrapCDMIMEX: explicit apply + CDM
update + prediction, interface products, implicit solve + correction) of the
256 x 128-cell perforated plate (p = 4, 24 holes, ~480k active DOFs, FP64).

Timing (device, CUDA events on the launching stream):
  * value: K steps, each timed alone, with the 129 MB L2 flushed (a 256 MB
    write) between steps, outside the timed events; the sum of the step times
    is the timed region.  Per-kernel times come from a second pass of as many
    flushed steps with an event between the explicit kernel and the solve
    chain as well (imex_step_profile).
  * warm: K consecutive steps without flushes (the state stays L2-resident,
    as in a long simulation).
  * e2e: the public host-I/O call (imex_step_io): every step uploads that
    step's source samples from pinned host memory and downloads the receiver
    trace (64 receivers) to pinned host memory; wall-clock time.
  * cpu_baseline: the CPU oracle (scipy.sparse + SuperLU, one core) on the same
    workload, a bounded number of steps after its untimed setup.
Under torchrun (N > 1) every rank runs an independent replica on its own GPU
(the method shards into independent problems; no data-path collective): the
timed region is bracketed by barriers and the max over ranks is taken.  The
batched workload's 64 source columns are split between the ranks
(replicas.shard_columns) and reported over the slowest rank's time.
"""
import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

os.environ.setdefault("OMP_NUM_THREADS", "1")
os.environ.setdefault("OPENBLAS_NUM_THREADS", "1")
os.environ.setdefault("MKL_NUM_THREADS", "1")

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "IMEX DOF-steps/s (FP64)"
UNIT = "DOF-steps/s"
# FP64 peak from unit counts and clocks (152 SMs x 2 DFMA/clk/SM x 2 flop x
# 2070 MHz), for context only: the roofline denominator is the FMA rate that
# imex_probe_fp64 measures in the same run (fp64_peak below).
FP64_PEAK_DERIVED_GFLOPS = 152 * 2 * 2 * 2.070
L2_FLUSH_BYTES = 256 << 20
# Kernels of one step in imex_step_profile's phase order (the third phase is
# the whole step): the explicit apply, and the implicit chain (walks + tops,
# the first walk also forming the right-hand sides).
PHASES = ("k_explicit2d", "k_walk+k_top")
# Explicit-apply variants of the setup autotuner (imex_info explicit_variant).
EXPLICIT_VARIANTS = ("tiles_large", "tiles_small", "sweep", "sweep_short", "tiles_large_split1",
                     "tiles_large_split2", "tiles_small_split2", "tiles_small_split4")


def phase_launches(st):
    """Launches per step of each phase of the per-phase pass: the explicit
    apply is one launch there (the split explicit launch runs only in plain
    steps, where it adds the far tiles' launch to launches_per_step), the
    solve chain is the rest of the step (forward walk, dense tops, backward
    walk, and more where there are more levels)."""
    xsplit = "split" in EXPLICIT_VARIANTS[st["explicit_variant"]]
    return {PHASES[0]: 1, PHASES[1]: max(1, int(st["launches_per_step"]) - (2 if xsplit else 1))}


def dominant_kernel(per_step_ms, launches):
    """The phase whose launches are longest on average: the roofline names a
    kernel, and the chain's phase is several launches."""
    return max(PHASES, key=lambda nm: per_step_ms[nm] / launches[nm])


def explicit_autotune_us(st):
    """Setup timing of every explicit candidate (one whole step, us; None: not timed)."""
    us = [st["explicit_tile_us_large"], st["explicit_tile_us_small"], st["explicit_sweep_us"],
          st["explicit_sweep_short_us"]] + list(st["explicit_split_us"])
    return {n: (v or None) for n, v in zip(EXPLICIT_VARIANTS, us)}


# ncu summaries that carry each phase's DRAM bytes per launch (see profiles/).
PROFILE_FILES = {"k_explicit2d": "k_explicit2d_plate256.md", "k_walk+k_top": "solve_kernels_plate256.md"}


def profiled_traffic(phase, workload):
    """DRAM bytes per launch from the committed ncu summary, or None.

    The figure holds only for the kernel sources it was captured from: the
    summary records their sha256 and any change to them yields None."""
    name = PROFILE_FILES.get(phase)
    if workload != "plate256" or name is None:
        return None
    try:
        text = open(os.path.join(ROOT, "profiles", name)).read()
    except OSError:
        return None
    vals = {}
    for line in text.splitlines():
        line = line.strip().lstrip("-").strip()
        for key in ("dram_bytes_per_launch", "source_sha256"):
            if line.startswith(key + ":"):
                vals[key] = line.split(":", 1)[1].strip()
    if len(vals) != 2:
        return None
    h = hashlib.sha256()
    for f in ("step_kernels.cuh", "kernels.cuh"):
        with open(os.path.join(ROOT, "paper_2310_14712_gb300", "csrc", f), "rb") as fh:
            h.update(fh.read())
    return int(vals["dram_bytes_per_launch"]) if h.hexdigest() == vals["source_sha256"] else None


def time_flushed(g, steps, stream, flush):
    """Device time (ms) of `steps` single steps, each after an L2 flush: CUDA
    events on the launching stream at the boundaries of each step only (an
    event between the kernels of a step would stop the programmatic overlap of
    the solve chain's staging with the explicit kernel)."""
    import torch
    evs = []
    for k in range(steps):
        flush.fill_(float(k))
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        g.step(1, stream)
        e1.record(stream)
        evs.append((e0, e1))
    torch.cuda.synchronize()
    return sum(a.elapsed_time(b) for a, b in evs)


def time_flushed_phases(g, steps, stream, flush):
    """Per-phase device time (ms) summed over `steps` flushed steps, with CUDA
    events before the explicit kernel, between it and the solve chain and after
    the chain (imex_step_profile).  The middle event serialises the two phases,
    so their sum exceeds the plain step time of time_flushed."""
    total = np.zeros(len(PHASES) + 1)
    for k in range(steps):
        flush.fill_(float(k))
        total += np.asarray(g.step_profile(1, stream))
    return total


def measure_batched(imex, workloads, steps, stream, flush, rank=0, ws=1, device=None):
    """Independent source columns against the single-source form on the same
    geometry: the 16x16-cell plate with 64 seeded sources (one per column).
    With ws ranks the 64 columns are split between them (replicas.shard_columns:
    contiguous blocks, no collective on the data path); the value is all 64
    columns over the slowest rank's time.  The single-column comparison runs
    on one rank only."""
    out = {}
    full = workloads.multisource(nsrc=64)
    for label, ncols in (("batched", 64), ("plain", 1)):
        if label == "plain" and ws > 1:
            continue
        w = workloads.multisource(nsrc=ncols)
        mine = shard_columns(ncols, rank, ws) if label == "batched" else range(ncols)
        if label == "batched":
            w.src_pos = full.src_pos[mine.start:mine.stop]
        g = imex.Imex.from_workload(w, ncols=len(mine))
        st = g.info()
        g.step(5)
        ms = reduce_max(time_flushed(g, steps, stream, flush), ws, device)
        n_act = st["n_d"] + st["n_c"]
        out[label] = {"value": n_act * ncols * steps / (ms * 1e-3), "ms_per_step": ms / steps,
                      "ncols": ncols, "explicit_variant": EXPLICIT_VARIANTS[st["explicit_variant"]],
                      "explicit_autotune_us": explicit_autotune_us(st),
                      "solve_col_block": st["solve_col_block"],
                      "solve_col_block_autotune_us": {str(1 << k): (v or None)
                                                      for k, v in enumerate(st["solve_col_block_us"])}}
        g.close()
    b = out["batched"]
    b.update({"workload": "multisource: [0,1]^2 minus a centred circle r=0.2, 16x16 cells, p=4, "
                          "64 seeded sources (Ricker f0=20), one per column",
              "unit": UNIT, "steps": steps, "l2": "flushed between timed steps",
              "columns_per_rank": [len(shard_columns(64, r, ws)) for r in range(ws)]})
    if "plain" in out:
        b.update({"plain_value": out["plain"]["value"], "plain_ms_per_step": out["plain"]["ms_per_step"],
                  "speedup_vs_plain": b["value"] / out["plain"]["value"]})
    return b


def snapshot(g):
    """State (u, u_{n-1} on I_d, v^c, a^c) and step counter of a context."""
    return ({k: g.fields(k, out=np.zeros(g.field_len)) for k in ("u", "u_prev_d", "v_c", "a_c")},
            g.info()["step"])


def restore(g, snap):
    for k, v in snap[0].items():
        g.set_fields(k, v)
    g.set_step(snap[1])


def measure_learned_pcg(imex, w, steps, stream, flush, epochs=300, lr=0.1, t_active=600, guess_steps=40):
    """The implicit solve by PCG (tol 1e-10) against the factorised solve on
    the bench workload, all from one snapshot taken after t_active steps,
    when the pulse has reached the holes (before that the implicit right-hand
    sides are exactly zero and PCG takes no iteration): the learned FSAI
    (Kaporin training on the GPU), the same with the starting guess learned
    from the method's own solutions, the closed-form FSAI of the pattern, and
    Jacobi."""
    g = imex.Imex.from_workload(w)
    st = g.info()
    n_act = st["n_d"] + st["n_c"]
    g.step(t_active - guess_steps)
    t0 = time.perf_counter()
    hist = g.pcg_train(epochs, lr)
    train_s = time.perf_counter() - t0
    g.set_solver("pcg_fsai", 1e-10, 5000)
    t0 = time.perf_counter()
    wts, ghist = g.pcg_train_guess(guess_steps, 300, 0.05)
    guess_s = time.perf_counter() - t0
    snap = snapshot(g)
    out = {"workload": workload_name(w), "unit": UNIT, "tol": 1e-10, "train_epochs": epochs, "lr": lr,
           "train_seconds": train_s, "kaporin_loss": [float(hist[0]), float(hist[-1])],
           "guess_weights": [float(x) for x in wts], "guess_train_steps": guess_steps,
           "guess_train_seconds": guess_s, "guess_loss": [float(ghist[0]), float(ghist[-1])],
           "l2": "flushed between timed steps", "steps": steps,
           "window": f"steps {t_active + 3}..{t_active + 3 + steps} from one snapshot"}

    def run(label, solver, guess):
        restore(g, snap)
        g.set_solver(solver, 1e-10, 5000)
        g.pcg_set_guess(guess)
        g.step(3)
        s0 = g.pcg_status()
        ms = time_flushed(g, steps, stream, flush)
        s1 = g.pcg_status()
        out[label] = {"value": n_act * steps / (ms * 1e-3), "ms_per_step": ms / steps,
                      "iterations_per_step": (s1["iters_total"] - s0["iters_total"]) / steps,
                      "fallbacks": s1["fallbacks"] - s0["fallbacks"]}

    run("direct", "direct", False)
    run("pcg_fsai", "pcg_fsai", False)
    run("pcg_fsai_guess", "pcg_fsai", True)
    g.pcg_fsai_closed_form()
    run("pcg_fsai_closed_form", "pcg_fsai", False)
    run("pcg_jacobi", "pcg_jacobi", False)
    out["learned_vs_jacobi_iterations"] = (out["pcg_fsai"]["iterations_per_step"] /
                                           max(out["pcg_jacobi"]["iterations_per_step"], 1e-30))
    out["guess_vs_plain_iterations"] = (out["pcg_fsai_guess"]["iterations_per_step"] /
                                        max(out["pcg_fsai"]["iterations_per_step"], 1e-30))
    out["trained_vs_closed_form_iterations"] = (out["pcg_fsai"]["iterations_per_step"] /
                                                max(out["pcg_fsai_closed_form"]["iterations_per_step"], 1e-30))
    out["learned_vs_direct_value"] = out["pcg_fsai_guess"]["value"] / out["direct"]["value"]
    g.close()
    return out


def measure_schemes(imex, workloads, steps, stream, flush):
    """The paper's comparison schemes against the method on the same
    discretisation, each at its own default step (0.9 x its cell-wise critical
    step): per-step time, and simulated time advanced per second of device
    time, which is what the schemes' different stable steps trade against.
    On the 256x128 plate the all-implicit trapezoidal scheme factorises all
    480k active DOFs (its largest supernodes are walked as row chunks over
    many CTAs)."""
    out = {"l2": "flushed between timed steps", "steps": steps, "unit": "DOF-steps/s"}
    for wname, w, names in (("plate16", workloads.plate16(), ("imex", "cdm", "cdm_hrz", "trapezoidal")),
                            ("plate256", workloads.plate256(), ("imex", "cdm", "cdm_hrz", "trapezoidal"))):
        res = {"workload": workload_name(w)}
        for sch in names:
            with imex.Imex.from_workload(w, scheme=sch) as g:
                st = g.info()
                n_act = st["n_d"] + st["n_c"]
                g.step(3)
                ms = time_flushed(g, steps, stream, flush)
            res[sch] = {"dt": st["dt"], "dt_crit_uncut": st["dt_crit_uncut"],
                        "dt_crit_cut_min": st["dt_crit_cut_min"] or None, "n_d": st["n_d"], "n_c": st["n_c"],
                        "ms_per_step": ms / steps, "value": n_act * steps / (ms * 1e-3),
                        "sim_time_per_s": st["dt"] * steps / (ms * 1e-3)}
        ref = res["imex"]["sim_time_per_s"]
        for sch in names:
            res[sch]["sim_time_vs_imex"] = res[sch]["sim_time_per_s"] / ref
        out[wname] = res
    return out


def measure_voids3d(imex, workloads, stream, flush, steps=10, epochs=300, lr=0.2, t_active=20):
    """The 3D voided solid at full size (64x64x32 cells, p=3, 40 ellipsoidal
    voids, octree depth 2): the factorised solve (nested-dissection Cholesky
    computed at setup; its supernodes reach 1732 rows and are walked as row
    chunks over many CTAs) against PCG to 1e-10 with the learned FSAI
    preconditioner (trained first) and with Jacobi, all three from one
    snapshot taken t_active steps in."""
    import time as _t
    w = workloads.voids3d()
    t0 = _t.perf_counter()
    g = imex.Imex.from_workload(w)
    setup_s = _t.perf_counter() - t0
    st = g.info()
    n_act = st["n_d"] + st["n_c"]
    out = {"workload": (f"voids3d: [0,1]x[0,1]x[0,0.5] minus {len(w.holes)} ellipsoids, "
                        f"{w.ncells[0]}x{w.ncells[1]}x{w.ncells[2]} cells, p={w.p}, alpha={w.alpha:g}, "
                        f"octree depth {w.depth}, Ricker f0={w.f0:g}"),
           "unit": UNIT, "n_nodes": st["n_nodes"], "n_d": st["n_d"], "n_c": st["n_c"], "n_cut": st["n_cut"],
           "n_uncut": st["n_uncut"], "nnz_L": st["nnz_L"], "max_block": st["max_block"],
           "large_supernodes": st["large_supernodes"], "solve_levels": st["solve_levels"],
           "components": st["n_components"], "dt": st["dt"], "factorized": st["factorized"],
           "setup_seconds": setup_s, "device_bytes": st["device_bytes"], "tol": 1e-10,
           "l2": "flushed between timed steps", "steps": steps}

    def timed(solver, nsteps):
        g.set_solver(solver, 1e-10, 5000)
        g.step(2)
        a = g.pcg_status()
        ph = [0.0, 0.0, 0.0]
        for k in range(nsteps):
            flush.fill_(float(k))
            for q, v in enumerate(g.step_profile(1, stream)):
                ph[q] += v
        b = g.pcg_status()
        P = w.p + 1
        return {"value": n_act * nsteps / (ph[2] * 1e-3), "ms_per_step": ph[2] / nsteps,
                "explicit_ms": ph[0] / nsteps, "implicit_ms": ph[1] / nsteps,
                "explicit_fp64_tflops": 14 * P ** 4 * st["n_uncut"] / (ph[0] / nsteps * 1e-3) / 1e12,
                "iterations_per_step": (b["iters_total"] - a["iters_total"]) / nsteps,
                "fallbacks": b["fallbacks"] - a["fallbacks"]}

    t0 = _t.perf_counter()
    hist = g.pcg_train(epochs, lr)
    out["train_epochs"] = epochs
    out["lr"] = lr
    out["train_seconds"] = _t.perf_counter() - t0
    out["kaporin_loss"] = [float(hist[0]), float(hist[-1])]
    g.set_solver("pcg_fsai", 1e-10, 5000)
    t0 = _t.perf_counter()
    wts, ghist = g.pcg_train_guess(t_active, 300, 0.05)
    out["guess_weights"] = [float(x) for x in wts]
    out["guess_train_steps"] = t_active
    out["guess_train_seconds"] = _t.perf_counter() - t0
    out["guess_loss"] = [float(ghist[0]), float(ghist[-1])]
    snap = snapshot(g)
    out["window"] = f"steps {t_active + 2}.. from one snapshot"

    def timed_guess(solver, nsteps, guess):
        restore(g, snap)
        g.pcg_set_guess(guess)
        return timed(solver, nsteps)

    out["direct"] = timed_guess("direct", steps, False)
    out["pcg_fsai"] = timed_guess("pcg_fsai", steps, False)
    out["pcg_fsai_guess"] = timed_guess("pcg_fsai", steps, True)
    out["pcg_jacobi"] = timed_guess("pcg_jacobi", max(2, steps // 2), False)
    t0 = _t.perf_counter()
    g.pcg_fsai_closed_form()
    out["closed_form_seconds"] = _t.perf_counter() - t0
    out["pcg_fsai_closed_form"] = timed_guess("pcg_fsai", steps, False)
    out["value"] = out["direct"]["value"]
    out["learned_vs_jacobi_iterations"] = (out["pcg_fsai"]["iterations_per_step"] /
                                           max(out["pcg_jacobi"]["iterations_per_step"], 1e-30))
    out["guess_vs_plain_iterations"] = (out["pcg_fsai_guess"]["iterations_per_step"] /
                                        max(out["pcg_fsai"]["iterations_per_step"], 1e-30))
    out["trained_vs_closed_form_iterations"] = (out["pcg_fsai"]["iterations_per_step"] /
                                                max(out["pcg_fsai_closed_form"]["iterations_per_step"], 1e-30))
    out["learned_vs_direct_value"] = out["pcg_fsai_guess"]["value"] / out["direct"]["value"]
    g.close()
    return out


def measure_adjoint(imex, workloads, nrec=64, checkpoint_every=100):
    """Misfit gradient in the per-cell wave speed by the discrete adjoint, on
    the adjoint workload (16x16-cell plate, smooth seeded speed, 16 sources as
    columns, 64 receivers, 2000 steps, checkpoint every 100), against the
    forward run of the same steps.  Host wall clock around the calls."""
    import numpy as np
    import torch
    w = workloads.adjoint()
    rec = workloads.receiver_nodes(w, nrec)
    ncols = len(w.src_pos)
    data = np.zeros((w.steps, ncols, nrec))
    out = {"workload": "adjoint: [0,1]^2 minus a centred circle r=0.2, 16x16 cells, p=4, per-cell "
                       f"speed in [0.8,1.2], {ncols} sources (columns), {nrec} receivers, "
                       f"{w.steps} steps, checkpoint every {checkpoint_every}",
           "unit": "s"}
    with imex.Imex.from_workload(w, ncols=ncols) as g:
        st = g.info()
        g.step(20)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        g.step(w.steps)
        torch.cuda.synchronize()
        out["forward_seconds"] = time.perf_counter() - t0
    with imex.Imex.from_workload(w, ncols=ncols) as g:
        g.adjoint(50, rec, data[:50], 10)          # warm-up (allocations, code paths)
    with imex.Imex.from_workload(w, ncols=ncols) as g:
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        J, grad = g.adjoint(w.steps, rec, data, checkpoint_every)
        out["gradient_seconds"] = time.perf_counter() - t0
    n_act = st["n_d"] + st["n_c"]
    out["gradient_over_forward"] = out["gradient_seconds"] / out["forward_seconds"]
    out["gradient_dof_steps_per_s"] = n_act * ncols * w.steps / out["gradient_seconds"]
    out["finite"] = bool(np.isfinite(J) and np.isfinite(grad).all())
    return out


def fp64_peak(imex):
    """FP64 pipe rates measured now by imex_probe_fp64 (independent FMA, add and
    multiply chains over every SM); the FMA rate x 2 flops is the peak."""
    h = hashlib.sha256()
    with open(os.path.join(ROOT, "paper_2310_14712_gb300", "csrc", "probe.cu"), "rb") as fh:
        h.update(fh.read())
    out = {"source": "paper_2310_14712_gb300/csrc/probe.cu", "source_sha256": h.hexdigest()}
    for kind in ("fma", "add", "mul"):
        rate, secs = imex.probe_fp64(kind, 40000)
        out[f"{kind}_lane_ops_per_s"] = rate
        out[f"{kind}_seconds"] = secs
    out["fma_tflops"] = 2.0 * out["fma_lane_ops_per_s"] / 1e12
    out["derived_tflops"] = FP64_PEAK_DERIVED_GFLOPS / 1e3
    return out


def measured_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f)
    except Exception:
        return {}


def algorithmic(st, P, Pd):
    """Per-launch algorithmic FP64 flops and HBM bytes of each kernel (one step)."""
    n_d, n_c, n_iface, n_cut, nnz = st["n_d"], st["n_c"], st["n_iface"], st["n_cut"], st["nnz_L"]
    n_uncut, n_nodes = st["n_uncut"], st["n_nodes"]
    # FP64 flops the explicit kernel executes per cell row / column item: the
    # stiffness in even-odd form and the mass as diagonal + rank one.
    H, odd = P // 2, P % 2
    x_item = 2 * H + H * (4 * H + 2 + odd) + odd * (1 + 2 * H) + (2 * H + odd) + 3 * P
    y_item = (4 * H + odd) + 2 * H + H * (4 * H + 2 + odd) + odd * (1 + 2 * H) + 4 * P
    return {
        # A1+A2: 4 contractions of P^3 FMAs per uncut cell (the plain sum
        # factorisation), ~10 flops per DOF update, prediction.
        "k_explicit2d": {"flops": 8 * P ** 3 * n_uncut + 10 * n_d + 4 * n_c,
                         "exec_flops": P * (x_item + y_item) * n_uncut + 10 * n_d + 4 * n_c,
                         "bytes": 8 * (4 * n_d + 2 * n_c) + n_nodes},
        # A4 (row-wise: one P^d dot product per (c-row, interface cell) pair),
        # A5 forward and backward substitution over the factor, A6 correction.
        "k_walk+k_top": {"flops": 2 * Pd * st["rhs_pairs"] + 4 * nnz + 10 * n_c,
                         "bytes": 8 * (Pd * Pd * n_cut + Pd * n_iface) + 2 * 12 * nnz + 8 * 6 * n_c},
    }


class ClockSampler:
    """nvidia-smi samples during the timed region (200 ms period)."""

    def __init__(self, index):
        self.proc = None
        self.path = None
        self.index = index

    def __enter__(self):
        try:
            fd, self.path = tempfile.mkstemp(suffix=".csv")
            os.close(fd)
            q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
                 "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
                 "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.index}", f"--query-gpu={q}", "--format=csv,noheader,nounits",
                 "-lms", "200"], stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
            time.sleep(0.3)
        except Exception:
            self.proc = None
        return self

    def __exit__(self, *a):
        if self.proc is not None:
            time.sleep(0.25)
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()

    def summary(self):
        if not self.path or not os.path.exists(self.path):
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        sm, smax, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            f = [x.strip() for x in line.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                smax = float(f[2])
            except ValueError:
                continue
            for nm, v in zip(names, f[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        os.unlink(self.path)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": smax,
                "reasons": sorted(reasons), "samples": len(sm)}


from paper_2310_14712_gb300.replicas import barrier, dist_env, reduce_max, shard_columns  # noqa: E402


def cpu_oracle_rate(w, nsteps, warmup=1):
    """Oracle steps per second on the host (setup untimed); returns (rate, n_active, seconds)."""
    from oracle import pipeline
    s = pipeline.setup(**w.kwargs())
    st = s.imex.initial_state()
    for _ in range(warmup):
        st = s.imex.step(st)
    t0 = time.perf_counter()
    for _ in range(nsteps):
        st = s.imex.step(st)
    dt = time.perf_counter() - t0
    n_act = int(s.disc.active.sum())
    return n_act * nsteps / dt, n_act, dt


def run_reference(args):
    ws, rank, _ = dist_env()
    if rank != 0:
        return 0
    from paper_2310_14712_gb300 import workloads
    w = workloads.get(args.workload)
    rate, n_act, secs = cpu_oracle_rate(w, args.steps, args.warmup)
    line = {
        "impl": "reference", "metric": METRIC, "value": rate, "unit": UNIT, "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * secs / max(args.steps, 1),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic",
        "config": {"workload": workload_name(w), "parallelism": "single CPU core"},
        "cpu_baseline": {"value": rate, "unit": UNIT, "cores": 1, "kind": "oracle",
                         "sample": f"{args.steps} oracle IMEX steps of {w.name} after {args.warmup} untimed"},
        "e2e": {"value": rate, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)
    return 0


def workload_name(w):
    box = "x".join(f"[{a:g},{b:g}]" for a, b in zip(w.lo, w.hi))
    return (f"{w.name}: {box} minus {len(w.holes)} circles, {w.ncells[0]}x{w.ncells[1]} cells, "
            f"p={w.p}, alpha={w.alpha:g}, quadtree depth {w.depth}, Ricker f0={w.f0:g}")


def run_gpu(args):
    import torch
    ws, rank, local = dist_env()
    if ws > 1:
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    else:
        torch.cuda.set_device(0)
    device = torch.device("cuda", torch.cuda.current_device())
    from paper_2310_14712_gb300 import imex, workloads
    w = workloads.get(args.workload)
    g = imex.Imex.from_workload(w)
    st = g.info()
    n_act = st["n_d"] + st["n_c"]
    P = w.p + 1
    Pd = P ** w.dim
    stream = torch.cuda.current_stream(device)
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device=device)

    # Warm-up (W steps, untimed).
    g.step(args.warmup)
    torch.cuda.synchronize()

    # Timed region: K steps, each alone between L2 flushes; events at the step
    # boundaries on the launching stream.
    barrier(ws)
    torch.cuda.synchronize()
    with ClockSampler(device.index) as clk:
        wall0 = time.perf_counter()
        t_step_ms = time_flushed(g, args.steps, stream, flush)
        wall = time.perf_counter() - wall0
    barrier(ws)
    t_max_ms = reduce_max(t_step_ms, ws, device)
    value = ws * n_act * args.steps / (t_max_ms * 1e-3)

    # Per-kernel times: the same number of flushed steps with events between
    # the explicit kernel and the solve chain as well.
    phase = time_flushed_phases(g, args.steps, stream, flush)

    # Warm (continuous) stepping, no flushes.
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    e0.record(stream)
    g.step(args.steps, stream)
    e1.record(stream)
    torch.cuda.synchronize()
    warm_ms = reduce_max(e0.elapsed_time(e1), ws, device)

    # End to end through the host-I/O entry point: source samples in, receiver traces out.
    ft = torch.from_numpy(workloads.source_signature(args.steps + 1, st["dt"])).pin_memory()
    rec = torch.from_numpy(workloads.receiver_nodes(w, 64)).pin_memory()
    traces = torch.zeros((args.steps, len(rec)), dtype=torch.float64).pin_memory()
    torch.cuda.synchronize()
    barrier(ws)
    t0 = time.perf_counter()
    g.step_io(args.steps, ft, rec, traces, stream)
    e2e_s = reduce_max(time.perf_counter() - t0, ws, device)
    e2e = {"value": ws * n_act * args.steps / e2e_s, "unit": UNIT,
           "h2d_bytes_per_step": 2 * 8, "d2h_bytes_per_step": 8 * int(len(rec)),
           "call": "imex_step_io: source samples H2D + 64 receiver samples D2H every step"}
    assert np.isfinite(traces.numpy()).all()

    fp64 = fp64_peak(imex)
    peak_gflops = fp64["fma_tflops"] * 1e3
    alg = algorithmic(st, P, Pd)
    per_launch_ms = {nm: phase[i] / args.steps for i, nm in enumerate(PHASES)}
    launches = phase_launches(st)
    dom = dominant_kernel(per_launch_ms, launches)
    peaks = measured_peaks()
    hbm = peaks.get("hbm_gbs")
    ach_gflops = alg[dom]["flops"] / (per_launch_ms[dom] * 1e-3) / 1e9
    xkern = "k_sweep2d" if st["explicit_variant"] in (2, 3) else "k_explicit2d"
    roof = {"kernel": xkern if dom == "k_explicit2d" else dom, "bound": "alu", "achieved": ach_gflops / 1e3, "peak": peak_gflops / 1e3,
            "unit": "TFLOP/s", "frac": ach_gflops / peak_gflops,
            "traffic": profiled_traffic(dom, args.workload), "traffic_unit": "bytes per launch (ncu)",
            "chosen_as": "longest mean launch in the per-phase pass (phase time per step / its launches per step)",
            "peak_source": ("measured in this run: imex_probe_fp64, independent FP64 FMA chains on every SM "
                            f"(csrc/probe.cu sha256 {fp64['source_sha256'][:16]}); of measured")}
    kernels = {}
    for nm in PHASES:
        t = per_launch_ms[nm] * 1e-3
        if t <= 0:
            continue
        kernels[nm] = {"ms": per_launch_ms[nm], "launches_per_step": launches[nm],
                       "share": per_launch_ms[nm] / (phase[len(PHASES)] / args.steps),
                       "fp64_tflops": alg[nm]["flops"] / t / 1e12,
                       "fp64_tflops_executed": alg[nm].get("exec_flops", alg[nm]["flops"]) / t / 1e12,
                       "fp64_frac": alg[nm]["flops"] / t / 1e9 / peak_gflops,
                       "hbm_gbs": alg[nm]["bytes"] / t / 1e9,
                       "hbm_frac": (alg[nm]["bytes"] / t / 1e9 / hbm) if hbm else None}
    clocks = clk.summary()
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": t_max_ms / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": workload_name(w), "n_active": n_act, "n_d": st["n_d"], "n_c": st["n_c"],
                   "n_nodes": st["n_nodes"], "components": st["n_components"], "nnz_L": st["nnz_L"],
                   "dt": st["dt"], "solve_levels": st["solve_levels"], "solve_ctas": st["solve_ctas"],
                   "solve_smem_bytes": st["solve_smem_bytes"],
                   "explicit_variant": EXPLICIT_VARIANTS[st["explicit_variant"]],
                   "explicit_autotune_us": explicit_autotune_us(st),
                   "explicit_autotune_basis": ("one whole step per candidate at setup (state restored), "
                                               "best over the walk launches' shared-memory requests"),
                   "solve_smem_request": st["solve_smem_bytes"], "solve_smem_needed": st["solve_smem_needed"],
                   "warm_kernel_ms": None,
                   "l2": "flushed (256 MB write) between timed steps",
                   "step_timing": "CUDA events on the launching stream at the boundaries of each timed step",
                   "kernel_timing": ("a second pass of as many flushed steps with an event between the explicit "
                                     "kernel and the solve chain as well (it stops their programmatic overlap; "
                                     f"{phase[len(PHASES)] / args.steps * 1e3:.1f} us per step in that pass)"),
                   "parallelism": f"replicas x{ws}" if ws > 1 else "1 GPU"},
        "roofline": roof,
        "roofline_hbm_view": {"kernel": dom, "achieved": kernels[dom]["hbm_gbs"], "peak": hbm, "unit": "GB/s",
                              "frac": kernels[dom]["hbm_frac"],
                              "step_frac": (sum(a["bytes"] for a in alg.values()) / (t_step_ms / args.steps * 1e-3)
                                            / 1e9 / hbm) if hbm else None},
        "kernels": kernels,
        "fp64_probe": fp64,
        "warm": {"value": ws * n_act * args.steps / (warm_ms * 1e-3), "ms_per_step": warm_ms / args.steps},
        "e2e": e2e,
        "clocks": clocks,
        "gpu_launches": st["launches_per_step"] * args.steps,
        "setup_seconds": st["setup_seconds"],
        "wall_seconds_timed_loop": wall,
    }
    if ws > 1 and not args.no_extras:   # the batched columns split across the ranks
        line["batched"] = measure_batched(imex, workloads, min(args.steps, 200), stream, flush, rank, ws, device)
    if ws == 1 and not args.no_extras:
        line["batched"] = measure_batched(imex, workloads, min(args.steps, 200), stream, flush)
        line["learned_pcg"] = measure_learned_pcg(imex, w, min(args.steps, 20), stream, flush)
        line["adjoint"] = measure_adjoint(imex, workloads)
        line["schemes"] = measure_schemes(imex, workloads, min(args.steps, 200), stream, flush)
        line["voids3d"] = measure_voids3d(imex, workloads, stream, flush)
    if rank == 0 and ws == 1 and not args.no_cpu_baseline:
        rate, n_act_cpu, secs = cpu_oracle_rate(w, args.cpu_steps)
        line["cpu_baseline"] = {"value": rate, "unit": UNIT, "cores": 1, "kind": "oracle",
                                "sample": f"{args.cpu_steps} oracle IMEX steps of {w.name} "
                                          f"(of {w.steps}), setup untimed, {secs:.1f} s"}
    if rank == 0:
        print(json.dumps(line), flush=True)
    g.close()
    if ws > 1:
        import torch.distributed as dist
        dist.destroy_process_group()
    return 0


def main():
    ap = argparse.ArgumentParser(description=__doc__.split("\n")[0])
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=2000)
    ap.add_argument("--warmup", type=int, default=20)
    ap.add_argument("--impl", default="gb300", choices=["gb300", "reference"])
    ap.add_argument("--workload", default="plate256")
    ap.add_argument("--cpu-steps", type=int, default=1000)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-extras", action="store_true",
                    help="only the headline measurement (no batched, PCG, adjoint or scheme lines)")
    args = ap.parse_args()
    if args.warmup < 3:
        ap.error("--warmup must be >= 3")
    if args.impl == "reference":
        return run_reference(args)
    return run_gpu(args)


if __name__ == "__main__":
    sys.exit(main())
