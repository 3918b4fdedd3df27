#!/usr/bin/env python
"""Benchmark of the pFFT matvec and preconditioned loop-basis GMRES on GB300.

Workload (default): 8 bond wires (Au, r = 12.5 um 16-gon, 2 mm, pitch 100 um,
40,192 triangles, 20,096 loops), pFFT grid 128 x 64 x 32, 16 log-spaced
frequencies 1 MHz - 10 GHz x 8 ports = 128 right-hand sides.

One step = one application of the preconditioned loop operator
z = P(w)^-1 A Z_b(w) A^T x to all 128 right-hand sides (mixed precision: FP32
grid, FFT, near field and preconditioner; double-float loop maps), i.e. 128 pFFT
matvecs.  `value` = matvecs per second over all ranks.  Beside it: the plain
FP64 form, GMRES time to a 1e-6 preconditioned residual (plain and mixed), the
roofline of the dominant stage (device time from CUDA events recorded on the
launching stream in a second timed run of the same step with stage timing on), an end-to-end number through host
buffers, clocks sampled during the timed region and the CPU oracle baseline.

--impl reference times the plain FP64 CPU oracle on a bounded sample of the
same workload (see cpu_oracle_rate).  Multi-GPU: independent replicas (the
method has no exchange step on one geometry); value sums all ranks.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

MEASURED = os.path.join(ROOT, "MEASURED_PEAKS.json")
PLAN_PARAMS = dict(order=3, near_factor=4.0, near_min_diam=2.0, n_touch=16, h0=0.0)


def workload(name):
    import synth
    w = synth.WORKLOADS[name]()
    m = w["mesh"]
    return w, m


def rhs_omegas(freqs, nports):
    return np.repeat(2 * np.pi * np.asarray(freqs), nports)


def peaks():
    if os.path.exists(MEASURED):
        with open(MEASURED) as f:
            d = json.load(f)
        return d["hbm_gbs"], d.get("bf16_tflops"), "measured"
    return 6800.0, 1900.0, "fallback"


# ------------------------------------------------------------------ algorithmic work per stage launch

FP32_LANES_PER_SM = 128      # FP32 FMA lanes per SM (4 sub-partitions x 32) on Blackwell


def sm_count():
    """SMs of the current device, read from the device (152 on a GB300)."""
    import torch
    return int(torch.cuda.get_device_properties(torch.cuda.current_device()).multi_processor_count)

# dram__bytes_read.sum + dram__bytes_write.sum of one launch from an ncu capture of the
# current kernel, with the number of grids (3 x right-hand sides) of that capture; the
# figure is scaled to a launch of the bench by grids.  Only kernels captured since their
# last change are listed.
MEASURED_TRAFFIC = {"fft_yz": (348.81e6, 48)}   # k_plane_conv<128, 64> (zero-pad pruned), 2 frequencies x 8 ports


def alu_peak_tflops(sm_mhz, nsm):
    """FP32 FMA peak of the CUDA cores: SMs x lanes x 2 flop x SM clock."""
    return nsm * FP32_LANES_PER_SM * 2 * sm_mhz * 1e6 / 1e12


def plane_flops(Ny, Nz, My, Mz):
    """Flops of one x-frequency plane of the (y, z) convolution, counted as
    5 n log2 n per complex FFT of length n over the lines that carry data: the
    forward z transforms of the Ny input rows (rows Ny..My-1 are zero), the
    forward y transforms of all Mz columns, the real kernel product (2 flops a
    point), the inverse y transforms of all columns, and the inverse z
    transforms of the Ny rows that are kept."""
    return (2 * Ny * 5 * Mz * np.log2(Mz) + 2 * Mz * 5 * My * np.log2(My) + 2 * My * Mz)


def stage_work(stage, c):
    """(bound, algorithmic amount per launch group, unit) of one stage.

    Bytes are the unique data a stage must move (each operand read once,
    each result written once); flops count the real multiply-adds of the
    block-sparse products (a 3x3 real block times a complex 3-vector = 18 FMA
    = 36 flop per right-hand side).  c: sizes of the workload and plan."""
    R, cb = c["R"], c["cb"]
    Ng, Nx, My, Mz, nt, nl = c["Ng"], c["Nx"], c["My"], c["Mz"], c["nt"], c["nl"]
    if stage == "fft_x_fwd":          # grid read, x-padded grid written
        return "hbm", 3 * R * (Ng + 2 * Ng) * cb, "B"
    if stage == "fft_yz":
        # per x-frequency plane (2 Nx of them per grid): plane_flops; the kernel is bound by
        # instruction issue on the FP32 pipe and shared memory (ncu), not by HBM (its bytes:
        # stage_bytes below)
        return "alu", 3 * R * 2 * Nx * plane_flops(My // 2, Mz // 2, My, Mz), "flop"
    if stage == "fft_x_inv":          # x-padded grid read, grid written
        return "hbm", 3 * R * (2 * Ng + Ng) * cb, "B"
    if stage == "project":
        # c_T read, node-ordered block records read, grid written
        return "hbm", R * nt * 3 * cb + c["n_pair"] * c["rec"] + (Ng + 1) * 8 + 3 * R * Ng * cb, "B"
    if stage == "interp":
        # regroup: potentials of the nodes in use read and written once; far gather (mixed
        # form): those potentials and the triangle-ordered blocks read, the far field written
        b = 2 * 3 * R * c["n_active"] * cb
        if c.get("mixed", True):
            b += 3 * R * c["n_active"] * cb + c["n_pair"] * c["rec"] + R * nt * 3 * cb
        return "hbm", b, "B"
    if stage == "near":
        if c.get("mixed", True) and R % 2 == 0 and R >= 96:
            # tensor cores (split tf32, even R from 96): the near 3x3 blocks times complex right-hand sides
            return "tensor", 36 * R * c["n_near"], "flop"
        return "alu", 36 * R * (c["n_near"] + c["n_pair"]), "flop"
    if stage == "loop_to_branch":
        return "hbm", R * nl * 16 + R * nt * 3 * cb, "B"
    if stage == "branch_to_loop":
        return "hbm", R * nt * 3 * 16 + R * nl * 16, "B"
    if stage == "precond_apply":
        return "hbm", 2 * R * nl * 16, "B"
    return None


def stage_bytes(stage, c):
    """Unique HBM bytes of a stage whose primary bound is not HBM, for the
    second roofline basis: the (y, z) planes read the x-transformed grids
    (2 N_g values per grid) and write them back."""
    if stage == "fft_yz":
        return 3 * c["R"] * 4 * c["Ng"] * c["cb"]
    return None


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled every 200 ms."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.hw_slowdown,"
         "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
         "clocks_event_reasons.sw_power_cap")

    def __init__(self, device_index):
        self.dev = device_index
        self.proc = None
        self.path = None

    def start(self):
        """Starts sampling and returns once the first sample is written, so that
        nvidia-smi's own start-up does not fall inside the timed region."""
        try:
            fd, self.path = tempfile.mkstemp(suffix=".csv")
            os.close(fd)
            self.fh = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.dev}", f"--query-gpu={self.Q}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=self.fh, stderr=subprocess.DEVNULL)
        except OSError:
            self.proc = None
            return
        t0 = time.time()
        while time.time() - t0 < 5.0 and self.proc.poll() is None:
            if os.path.getsize(self.path) > 0:
                break
            time.sleep(0.02)

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        self.fh.close()
        rows = []
        with open(self.path) as f:
            for line in f:
                parts = [x.strip() for x in line.split(",")]
                if len(parts) >= 8:
                    rows.append(parts)
        os.unlink(self.path)
        if not rows:
            return None
        sm = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in rows for i in range(4) if r[4 + i].lower().startswith("active")})
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(rows)}


def shard(units, rank, world, sizes=None):
    """The units (independent geometries, or frequencies) rank `rank` of `world`
    processes.  With sizes: largest first, each to the least-loaded rank so far
    (ties to the lower rank), in the units' original order within a rank;
    without: every world-th unit from the rank on."""
    units = list(units)
    if sizes is None:
        return units[rank::world]
    load = [0.0] * world
    owner = [0] * len(units)
    for i in sorted(range(len(units)), key=lambda i: (-sizes[i], i)):
        r = min(range(world), key=lambda q: (load[q], q))
        owner[i] = r
        load[r] += sizes[i]
    return [u for u, o in zip(units, owner) if o == rank]


def aggregate(local_seconds, local_units, dist):
    """Whole-job throughput: units of all ranks / the slowest rank's time."""
    if dist is None:
        return local_units / local_seconds, local_seconds
    import torch
    t = torch.tensor([local_seconds], dtype=torch.float64)
    u = torch.tensor([local_units], dtype=torch.float64)
    dev = "cuda" if torch.cuda.is_available() and dist.get_backend() == "nccl" else "cpu"
    t, u = t.to(dev), u.to(dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    dist.all_reduce(u, op=dist.ReduceOp.SUM)
    return float(u.item()) / float(t.item()), float(t.item())


# ------------------------------------------------------------------ CPU oracle baseline

def cpu_oracle_rate(name, steps=1, warmup=0):
    """Plain FP64 oracle pFFT matvec (oracle.pfft, unchanged) on a bounded sample.

    The oracle's set-up for the full array is minutes of CPU; the sample is one
    of the array's wires (its first conductor) on the full array's grid, so the
    FFT convolution is the full-size one.  Per right-hand side:
      t(full) = t_fft + (wires) * (t_sample - t_fft)
    (projection, interpolation, near field, Gram and loop maps grow with the
    triangle count; the FFT part does not)."""
    import synth
    from synth.meshes import Mesh
    from oracle.graph import build_loops
    from oracle.pfft import PfftSystem, PfftParams
    w, m = workload(name)
    ncond = m.ncond
    if ncond > 1:
        keep = np.nonzero(m.cond == 0)[0]
        vmap = -np.ones(m.nv, np.int64)
        used = np.unique(m.tri[keep])
        vmap[used] = np.arange(used.shape[0])
        sub = Mesh(xyz=m.xyz[used], tri=vmap[m.tri[keep]].astype(np.int32), cond=np.zeros(keep.shape[0], np.int32),
                   sigma=m.sigma[:1], ports=[m.ports[0]])
    else:
        sub = m
    O = build_loops(sub)
    box = m.bbox()   # the full array's box: the sample's FFT is the full-size one
    params = PfftParams(grid=w["grid"], box=box, **{k: v for k, v in PLAN_PARAMS.items() if k != "h0"})
    S = PfftSystem(sub, O, params)
    x = synth.complex_gaussian(O.nl, 1, seed=7)[0]
    om = 2 * np.pi * 1e9
    for _ in range(warmup):
        S.matvec(x, om)
    t_mv, t_fft = [], []
    for _ in range(max(1, steps)):
        t0 = time.perf_counter()
        S.matvec(x, om)
        t_mv.append(time.perf_counter() - t0)
        g = np.zeros((3,) + tuple(S.op.N), complex)
        t0 = time.perf_counter()
        for c in range(3):
            S.op.convolve(g[c])
        t_fft.append(time.perf_counter() - t0)
    tm, tf = float(np.median(t_mv)), float(np.median(t_fft))
    wires = max(1, ncond)
    t_full = tf + wires * max(tm - tf, 0.0)
    sample = (f"conductor 0 of {wires} ({sub.nt} triangles, {O.nl} loops) on the full "
              f"{'x'.join(map(str, w['grid']))} grid, 1 RHS at 1 GHz; full-array time per RHS = "
              f"t_fft + {wires} x (t_sample - t_fft); t_sample = {tm:.3f} s, t_fft = {tf:.3f} s")
    return 1.0 / t_full, sample, t_full


# ------------------------------------------------------------------ main

def batch_main(args, ws, dist=None, n_total=None):
    """Batched uneven geometries: one step = one product of every plan's loop
    operator on its right-hand sides (all frequencies x ports of every
    geometry), through sie_batch_matvec replaying a captured CUDA graph; beside
    it the same batch launched eagerly on per-plan streams, and the plans one
    after another on one stream (pfft_matvec), all mixed; and FP64 eager."""
    import torch
    from paper_2210_04891_gb300 import api, SPACE_LOOP, PREC_FP64, PREC_MIXED, REFINE_OFF, REFINE_FP64, REFINE_DF
    import synth
    plans, xs, oms = [], [], []
    for k, w in enumerate(ws):
        m = w["mesh"]
        M = api.Mesh.from_synth(m)
        L = api.Loops(M, m.ports)
        plans.append(api.Plan(M, L, dict(PLAN_PARAMS, n_touch=8, grid=w["grid"])))
        om = rhs_omegas(w["freqs"], len(m.ports))
        oms.append(om)
        xs.append(torch.from_numpy(synth.complex_gaussian(L.nl, om.size, seed=100 + k)).cuda())
    B = api.Batch(plans)
    outs = [torch.empty_like(x) for x in xs]
    R = sum(int(x.shape[0]) for x in xs)
    stream = torch.cuda.current_stream()
    K, W = args.steps, max(3, args.warmup)

    def run(fn, K, W):
        for _ in range(W):
            fn()
        torch.cuda.synchronize()
        if dist:
            dist.barrier()
        l0 = sum(p.launches() for p in plans)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(K):
            fn()
        e1.record(stream)
        torch.cuda.synchronize()
        if dist:
            dist.barrier()
        return e0.elapsed_time(e1) / 1e3, sum(p.launches() for p in plans) - l0

    sampler = ClockSampler(int(os.environ.get("LOCAL_RANK", "0")))
    B.matvec(xs, oms, SPACE_LOOP, PREC_MIXED, graph=True, outs=outs)
    sampler.start()
    t_graph, launches = run(lambda: B.matvec(xs, oms, SPACE_LOOP, PREC_MIXED, graph=True, outs=outs), K, W)
    clocks = sampler.stop()
    t_eager, _ = run(lambda: B.matvec(xs, oms, SPACE_LOOP, PREC_MIXED, graph=False, outs=outs), K, W)

    def sequential():
        for p, x, o, y in zip(plans, xs, oms, outs):
            api.pfft_matvec(p, x, o, SPACE_LOOP, PREC_MIXED, out=y)
    t_seq, _ = run(sequential, K, W)
    K64 = max(3, K // 3)
    t_64, _ = run(lambda: B.matvec(xs, oms, SPACE_LOOP, PREC_FP64, graph=False, outs=outs), K64, 2)
    # whole-job rates: right-hand sides of all ranks over the slowest rank's time
    v_graph, t_graph = aggregate(t_graph, R * K, dist)
    v_eager, t_eager = aggregate(t_eager, R * K, dist)
    v_seq, t_seq = aggregate(t_seq, R * K, dist)
    v_64, t_64 = aggregate(t_64, R * K64, dist)
    R_all = int(round(aggregate(1.0, R, dist)[0]))
    gm = None
    if args.gmres_freqs > 0 and dist is None:
        # a first batched solve at other frequencies loads the solve kernels and builds each
        # plan's symbolic preconditioner; the timed solve then factors its own frequencies
        sel = np.linspace(0, len(ws[0]["freqs"]) - 1, args.gmres_freqs).astype(int)
        warm = [w["freqs"][np.clip(sel + 1, 0, len(w["freqs"]) - 1)] for w in ws]
        fr = [w["freqs"][sel] for w in ws]
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        B.solve(warm, tol=1e-6, restart=200, max_iter=1000, prec=PREC_MIXED)
        t_first = time.perf_counter() - t0
        t0 = time.perf_counter()
        res = B.solve(fr, tol=1e-6, restart=200, max_iter=1000, prec=PREC_MIXED, refine=REFINE_DF, graph=True)
        dt = time.perf_counter() - t0
        r0 = B.stats()["replays"]
        t0 = time.perf_counter()
        res_t = B.solve(fr, tol=1e-6, restart=200, max_iter=1000, prec=PREC_MIXED, refine=REFINE_DF)
        dt_t = time.perf_counter() - t0
        gm = {"tol": 1e-6, "form": "mixed with refinement (double-float residual products)", "seconds": dt,
              "step": "one CUDA graph replay per Arnoldi step of all plans (sie_batch_solve_graph)",
              "solves": int(sum(len(f) for f in fr)),
              "iterations_max": int(max(st["iterations_max"] for _, st in res)),
              "converged": bool(all(st["converged"] for _, st in res)),
              "equal_to_threaded": bool(all(np.array_equal(a[0], b[0]) for a, b in zip(res, res_t))),
              "threaded_seconds": dt_t,
              "includes": "per-frequency factorisations of every plan's preconditioner",
              "first_solve_seconds": t_first}
        del r0
    learned = None
    if args.learned_eval > 0 and dist is None:
        # train the correction on the first geometries' features and probing targets at
        # 1 and 10 GHz, then solve the held-out ones with the plain and the learned form
        ntrain = min(args.learned_eval, len(plans) - 1)
        eval_f = np.array([1e9, 1e10])
        feats, targets = [], []
        for k in range(ntrain):
            for j, f in enumerate(eval_f):
                alpha = torch.from_numpy(synth.complex_gaussian(plans[k].nb, 4, seed=500 + 2 * k + j)).cuda()
                feats.append(api.branch_features(plans[k], 2 * np.pi * f))
                targets.append(api.branch_probe_target(plans[k], alpha, 2 * np.pi * f))
        net = api.MLP(32, seed=1)
        t0 = time.perf_counter()
        losses = net.train(torch.cat(feats), torch.cat(targets), 400, lr=3e-3)
        torch.cuda.synchronize()
        t_train = time.perf_counter() - t0
        held = plans[ntrain:]
        Bh = api.Batch(held)
        fr = [eval_f] * len(held)
        Bh.solve([eval_f * 1.01] * len(held), tol=1e-6, restart=200, max_iter=1000, prec=PREC_MIXED)   # warm-up
        out = {}
        for name, m in (("plain", None), ("learned", net)):
            for p_ in held:
                api.set_learned(p_, m)
            t0 = time.perf_counter()
            res = Bh.solve(fr, tol=1e-6, restart=200, max_iter=1000, prec=PREC_MIXED)
            out[name] = {"seconds": time.perf_counter() - t0,
                         "iterations_sum": int(sum(st["iterations_sum"] for _, st in res)),
                         "iterations_max": int(max(st["iterations_max"] for _, st in res)),
                         "converged": bool(all(st["converged"] for _, st in res))}
            Zs = [Z for Z, _ in res]
            if name == "plain":
                Zp = Zs
            else:
                out[name]["Z_rel_vs_plain"] = float(max(np.abs(a - b).max() / np.abs(b).max() for a, b in zip(Zs, Zp)))
        for p_ in held:
            api.set_learned(p_, None)
        learned = {"train_geometries": ntrain, "held_out_geometries": len(held), "frequencies_hz": eval_f.tolist(),
                   "train_steps": 400, "train_seconds": t_train, "loss_first": float(losses[0]),
                   "loss_last": float(losses[-1]), **out,
                   "chosen": judge_learned(out)}
    world = dist.get_world_size() if dist else 1
    if dist and dist.get_rank() != 0:
        return
    line = {"metric": "pFFT matvecs/s (batched uneven geometries)", "value": v_graph, "unit": "matvec/s",
            "n_gpus": world, "steps": K, "warmup": W, "ms_per_step": 1e3 * t_graph / K, "higher_is_better": True,
            "scaling": "strong", "vs_baseline": None, "dtype": "f32+f64", "data": "synthetic",
            "config": {"workload": args.workload, "geometries": n_total or len(ws),
                       "geometries_on_rank0": len(ws),
                       "triangles_on_rank0": int(sum(w["mesh"].nt for w in ws)),
                       "loops_on_rank0": int(sum(p.nl for p in plans)), "rhs_per_step": R_all,
                       "step": "y_i = A Z_b A^T x_i for every geometry i (mixed), one graph launch per rank",
                       "parallelism": "geometries sharded over %d ranks (no exchange)" % world},
            "eager_streams": {"value": v_eager, "unit": "matvec/s", "ms_per_step": 1e3 * t_eager / K},
            "sequential_one_stream": {"value": v_seq, "unit": "matvec/s", "ms_per_step": 1e3 * t_seq / K},
            "plain_fp64": {"value": v_64, "unit": "matvec/s", "ms_per_step": 1e3 * t_64 / K64},
            "gmres_batched": gm, "learned_preconditioner": learned, "graph_stats": B.stats(), "clocks": clocks,
            "gpu_launches": launches}
    print(json.dumps(line))


LEARNED_MIN_GAIN = 0.02


def judge_learned(out):
    """The plain preconditioner judges the learned one: the learned form is kept
    only when it saves at least 2% of the GMRES iterations on the held-out set
    and leaves no more solves unconverged; otherwise the plain P is the fallback."""
    p, l = out["plain"], out["learned"]
    gain = 1.0 - l["iterations_sum"] / max(1, p["iterations_sum"])
    if gain >= LEARNED_MIN_GAIN and l.get("not_converged", 0) <= p.get("not_converged", 0):
        return "learned"
    return "plain (fallback: %.2f%% fewer iterations, below the %.0f%% bar)" % (100 * gain, 100 * LEARNED_MIN_GAIN)


def learned_main(args):
    """The learned preconditioner correction at its configured scale: a 6 -> 128 ->
    128 -> 1 network computing with FP16 weights and FP32 accumulation, trained on
    the device on features and probing targets of `learned_train` seeded geometries
    (meanders and bond-wire arrays, 5k-40k triangles; 256 branches sampled per
    geometry and frequency) at 1 and 10 GHz, then judged by the plain
    preconditioner on `learned_held_out` held-out geometries: mixed GMRES with
    refinement to 1e-6, iterations and time of both forms."""
    import torch
    from paper_2210_04891_gb300 import api, PREC_MIXED, REFINE_DF
    import synth
    torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", "0")))
    freqs = np.array([1e9, 1e10])
    per = 256
    gen = torch.Generator(device="cuda")
    gen.manual_seed(0)
    feats, targets = [], []
    t0 = time.perf_counter()
    ntri = 0
    for k in range(args.learned_train):
        w = synth.learned_geometry(1000 + k)
        m = w["mesh"]
        ntri += m.nt
        M = api.Mesh.from_synth(m)
        L = api.Loops(M, m.ports)
        P = api.Plan(M, L, dict(PLAN_PARAMS, n_touch=8, grid=w["grid"]))
        sel = torch.randint(0, P.nb, (per,), generator=gen, device="cuda")
        for j, f in enumerate(freqs):
            alpha = torch.from_numpy(synth.complex_gaussian(P.nb, 4, seed=100000 + 2 * k + j)).cuda()
            feats.append(api.branch_features(P, 2 * np.pi * f)[sel])
            targets.append(api.branch_probe_target(P, alpha, 2 * np.pi * f)[sel])
        del P, L, M
    torch.cuda.synchronize()
    t_data = time.perf_counter() - t0
    F, T = torch.cat(feats), torch.cat(targets)
    net = api.MLP(128, seed=1)
    t0 = time.perf_counter()
    losses = net.train(F, T, args.learned_steps, lr=1e-3)
    torch.cuda.synchronize()
    t_train = time.perf_counter() - t0
    out = {"plain": {"iterations_sum": 0, "seconds": 0.0, "not_converged": 0},
           "learned": {"iterations_sum": 0, "seconds": 0.0, "not_converged": 0}}
    zdiff, better, worse, ntri_eval = 0.0, 0, 0, 0
    for k in range(args.learned_held_out):
        w = synth.learned_geometry(5000 + k)
        m = w["mesh"]
        ntri_eval += m.nt
        M = api.Mesh.from_synth(m)
        L = api.Loops(M, m.ports)
        P = api.Plan(M, L, dict(PLAN_PARAMS, n_touch=8, grid=w["grid"]))
        its = {}
        for name in ("plain", "learned"):
            api.set_learned(P, net if name == "learned" else None)
            torch.cuda.synchronize()
            t1 = time.perf_counter()
            Z, st = api.sie_solve(P, freqs, tol=1e-6, restart=100, max_iter=500, prec=PREC_MIXED, refine=REFINE_DF)
            out[name]["seconds"] += time.perf_counter() - t1
            out[name]["iterations_sum"] += int(st["iterations_sum"])
            out[name]["not_converged"] += int(not st["converged"])
            its[name] = st["iterations_sum"]
            if name == "plain":
                Zp = Z
            else:
                zdiff = max(zdiff, float(np.abs(Z - Zp).max() / np.abs(Zp).max()))
        api.set_learned(P, None)
        better += its["learned"] < its["plain"]
        worse += its["learned"] > its["plain"]
        del P, L, M
    line = {"metric": "learned preconditioner correction: GMRES iterations and time to 1e-6, plain vs learned",
            "value": out["plain"]["iterations_sum"] / max(1, out["learned"]["iterations_sum"]),
            "unit": "plain / learned iterations", "higher_is_better": True, "data": "synthetic",
            "config": {"workload": "learned_%dx_5k-40k" % args.learned_train,
                       "network": "6 -> 128 -> 128 -> 1, tanh, FP16 weights, FP32 accumulation",
                       "train_geometries": args.learned_train, "train_triangles": ntri,
                       "samples": int(F.shape[0]), "branches_per_geometry_and_frequency": per,
                       "held_out_geometries": args.learned_held_out, "held_out_triangles": ntri_eval,
                       "frequencies_hz": freqs.tolist(), "solve": "mixed GMRES with FP64 refinement, tol 1e-6"},
            "data_seconds": t_data, "train_steps": args.learned_steps, "train_seconds": t_train,
            "loss_first": float(losses[0]), "loss_last": float(losses[-1]), **out,
            "held_out_fewer_iterations": better, "held_out_more_iterations": worse,
            "Z_rel_learned_vs_plain": zdiff,
            "chosen": judge_learned(out)}
    print(json.dumps(line))


def plane_pair_line(no_gmres):
    """The plane pair (517k triangles, grid 256 x 256 x 32, 8 frequencies x 4 ports = 32
    right-hand sides) measured in the same run as the headline: its mixed step (matvec +
    the nested-dissection P^-1), its FP64 step and, unless no_gmres, its mixed GMRES to 1e-6
    with double-float refinement residuals."""
    import torch
    import synth
    from paper_2210_04891_gb300 import api, SPACE_LOOP, PREC_FP64, PREC_MIXED, REFINE_DF
    t0 = time.perf_counter()
    w = synth.WORKLOADS["pdn_2x10mm_500k"]()
    m = w["mesh"]
    M = api.Mesh.from_synth(m)
    L = api.Loops(M, m.ports)
    P = api.Plan(M, L, dict(PLAN_PARAMS, grid=w["grid"]))
    freqs = w["freqs"]
    R = len(freqs) * len(m.ports)
    om = rhs_omegas(freqs, len(m.ports))
    x = torch.from_numpy(synth.complex_gaussian(L.nl, R, seed=7)).cuda()
    y, z = torch.empty_like(x), torch.empty_like(x)
    stream = torch.cuda.current_stream()

    def step(prec):
        api.pfft_matvec(P, x, om, SPACE_LOOP, prec, out=y)
        api.pfft_precond_apply(P, y, om, out=z, prec=prec)

    def timed(prec, K, W):
        for _ in range(W):
            step(prec)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(K):
            step(prec)
        e1.record(stream)
        torch.cuda.synchronize()
        return e0.elapsed_time(e1) / 1e3 / K

    t_mixed = timed(PREC_MIXED, 5, 3)     # the first warm-up step factors P for the 8 frequencies
    t_plain = timed(PREC_FP64, 2, 1)
    info = P.info()
    out = {"workload": w["name"], "triangles": int(m.nt), "loops": int(L.nl), "grid": list(w["grid"]),
           "rhs_per_step": R, "near_pairs": info["n_near_pairs"],
           "step": "z = P^-1 A Z_b A^T x (mixed; P^-1 by nested dissection)",
           "mixed": {"value": R / t_mixed, "unit": "matvec/s", "ms_per_step": 1e3 * t_mixed},
           "plain_fp64": {"value": R / t_plain, "unit": "matvec/s", "ms_per_step": 1e3 * t_plain}}
    if not no_gmres:
        torch.cuda.synchronize()
        t1 = time.perf_counter()
        Z, st = api.sie_solve(P, freqs, tol=1e-6, restart=100, max_iter=400, prec=PREC_MIXED, refine=REFINE_DF)
        out["gmres_mixed_refined_df"] = {"tol": 1e-6, "seconds": time.perf_counter() - t1,
                                         "iterations_max": st["iterations_max"], "converged": st["converged"],
                                         "residual_max": st["residual_max"]}
    out["wall_s"] = time.perf_counter() - t0
    del P
    return out


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=30)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="bondwires_8x2mm_40k")
    ap.add_argument("--no-gmres", action="store_true")
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--nfreq", type=int, default=0, help="use only the first N frequencies (profiling runs)")
    ap.add_argument("--step", default="matvec+precond", choices=["matvec+precond", "matvec"],
                    help="what one step applies (matvec: the plane pair, whose band preconditioner is too wide)")
    ap.add_argument("--gmres-freqs", type=int, default=0, help="batched workloads: frequencies per geometry solved")
    ap.add_argument("--learned-eval", type=int, default=0,
                    help="batched workloads: train the learned preconditioner correction on this many geometries "
                         "and compare it with the plain preconditioner on the others")
    ap.add_argument("--no-lossy", dest="lossy", action="store_false",
                    help="skip the lossy-kernel variant's timing")
    ap.add_argument("--learned-train", type=int, default=2000,
                    help="workload learned_c5: training geometries")
    ap.add_argument("--learned-held-out", type=int, default=200,
                    help="workload learned_c5: held-out geometries")
    ap.add_argument("--learned-steps", type=int, default=400, help="workload learned_c5: Adam steps")
    ap.add_argument("--no-plane-pair", dest="plane_pair", action="store_false",
                    help="default workload: skip the plane pair measured beside the headline")
    ap.add_argument("--graph", action="store_true",
                    help="with --step matvec: replay the product as a captured CUDA graph (a batch of one plan)")
    args = ap.parse_args()
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    import synth
    if args.workload == "learned_c5":
        if args.impl == "reference":
            print(json.dumps({"impl": "reference", "unavailable": "the oracle baseline covers single geometries"}))
            return
        if rank == 0:
            learned_main(args)
        return
    wl = synth.WORKLOADS[args.workload]()
    if isinstance(wl, list):
        if args.impl == "reference":
            print(json.dumps({"impl": "reference", "unavailable": "the oracle baseline covers single geometries"}))
            return
        import torch
        dist = None
        if world > 1:
            import torch.distributed as tdist
            tdist.init_process_group("nccl")
            dist = tdist
        torch.cuda.set_device(local)
        batch_main(args, shard(wl, rank, world, sizes=[w["mesh"].nt for w in wl]), dist, n_total=len(wl))
        if dist:
            dist.destroy_process_group()
        return
    w, m = workload(args.workload)
    freqs = w["freqs"][:args.nfreq] if args.nfreq > 0 else w["freqs"]
    nports = len(m.ports)
    R = len(freqs) * nports
    metric = "pFFT matvecs/s; GMRES time-to-1e-6 residual, plain vs mixed/learned form"

    if args.impl == "reference":
        if rank != 0:
            return
        from oracle.graph import build_loops
        nthreads = os.cpu_count()
        t0 = time.perf_counter()
        rate, sample, t_full = cpu_oracle_rate(args.workload, steps=args.steps, warmup=args.warmup)
        wall = time.perf_counter() - t0
        line = {"impl": "reference", "metric": metric, "value": rate, "unit": "matvec/s", "n_gpus": 0,
                "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * t_full,
                "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
                "data": "synthetic",
                "config": {"workload": w["name"], "triangles": int(m.nt), "loops": int(build_loops(m).nl),
                           "grid": list(w["grid"]), "rhs_per_step": 1, "frequencies": len(freqs), "ports": nports,
                           "step": "y = A Z_b A^T x (FP64 oracle, one right-hand side per step)",
                           "parallelism": "host cores"},
                "cpu_baseline": {"value": rate, "unit": "matvec/s", "cores": nthreads, "kind": "oracle",
                                 "sample": sample},
                "e2e": {"value": rate, "unit": "matvec/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
                "wall_s": wall}
        print(json.dumps(line))
        return

    import torch
    import torch.distributed as tdist
    dist = None
    if world > 1:
        tdist.init_process_group("nccl")
        dist = tdist
    torch.cuda.set_device(local)
    from paper_2210_04891_gb300 import api, SPACE_LOOP, PREC_FP64, PREC_MIXED, REFINE_OFF, REFINE_FP64, REFINE_DF

    M = api.Mesh.from_synth(m)
    L = api.Loops(M, m.ports)
    P = api.Plan(M, L, dict(PLAN_PARAMS, grid=w["grid"]))
    info = P.info()
    om = rhs_omegas(freqs, nports)
    import synth
    x = torch.from_numpy(synth.complex_gaussian(L.nl, R, seed=7)).cuda()
    y = torch.empty_like(x)
    z = torch.empty_like(x)
    stream = torch.cuda.current_stream()

    if args.step == "matvec":
        z = y          # the step's result is the product itself
    if args.graph and args.step != "matvec":
        raise SystemExit("--graph replays the product alone: use it with --step matvec")
    Bg = api.Batch([P]) if args.graph else None

    def step(prec):
        if Bg is not None:
            Bg.matvec([x], [om], SPACE_LOOP, prec, graph=True, outs=[y])
        else:
            api.pfft_matvec(P, x, om, SPACE_LOOP, prec, out=y)
        if args.step != "matvec":
            api.pfft_precond_apply(P, y, om, out=z, prec=prec)

    def timed(prec, K, W, profile=False):
        for _ in range(W):
            step(prec)
        torch.cuda.synchronize()
        if dist:
            dist.barrier()
        l0 = P.launches()
        if profile:
            P.profile(True)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        e0.record(stream)
        for _ in range(K):
            step(prec)
        e1.record(stream)
        torch.cuda.synchronize()
        if dist:
            dist.barrier()
        prof = P.profile_read() if profile else None
        if profile:
            P.profile(False)
        return e0.elapsed_time(e1) / 1e3, P.launches() - l0, prof

    K, W = args.steps, max(3, args.warmup)
    # mixed form: the headline
    sampler = ClockSampler(local)
    step(PREC_MIXED)
    torch.cuda.synchronize()
    sampler.start()
    t_mixed, launches, _ = timed(PREC_MIXED, K, W)
    clocks = sampler.stop()
    # stage split: a separate run with stage timing, so that the events it records stay
    # out of the headline's timed region
    Kp = max(3, K // 3)
    _, _, prof = timed(PREC_MIXED, Kp, 2, profile=True)
    value, tmax = aggregate(t_mixed, R * K, dist)
    # plain FP64 form
    t_plain, _, _ = timed(PREC_FP64, max(3, K // 3), 2)
    value_plain, _ = aggregate(t_plain, R * max(3, K // 3), dist)

    # roofline of the dominant stage
    hbm, bf16, src = peaks()
    Nx, Ny, Nz = w["grid"]
    from paper_2210_04891_gb300 import native as N
    pnode = P.export(N.EXPORT_PROJ_NODE)
    ctx = dict(R=R, cb=8, rec=48, Ng=Nx * Ny * Nz, Nx=Nx, My=2 * Ny, Mz=2 * Nz, nt=info["n_tri"], nl=L.nl,
               n_near=info["n_near_pairs"], n_pair=int(pnode.size), n_active=int(np.unique(pnode).size))
    timed_stages = [s for s in prof if prof[s][1] > 0]   # none when the step is a graph replay
    dom = max(timed_stages, key=lambda s: prof[s][0]) if timed_stages else None
    ms_dom, n_dom = prof[dom] if dom else (0.0, 0)
    stage_table = {s: {"ms_per_step": v[0] / Kp, "launch_groups": v[1]} for s, v in prof.items() if v[1]}
    roofline = None
    work = stage_work(dom, ctx) if dom else None
    if work:
        bound, amount, unit = work
        sec = ms_dom / n_dom / 1e3
        if bound == "hbm":
            achieved, peak, u, psrc = amount / sec / 1e9, hbm, "GB/s", src
        elif bound == "tensor":
            # tf32 dense peak = measured bf16 burst peak x nominal tf32/bf16 ratio (1.1 / 2.25 PFLOP/s)
            achieved, peak, u = amount / sec / 1e12, (bf16 or 1900.0) * 1.1 / 2.25, "TFLOP/s"
            psrc = f"{src} bf16 x 1.1/2.25 (tf32 nominal ratio)"
        else:
            mhz = (clocks or {}).get("sm_max_mhz") or 2070.0
            nsm = sm_count()
            achieved, peak, u = amount / sec / 1e12, alu_peak_tflops(mhz, nsm), "TFLOP/s"
            psrc = (f"derived: {nsm} SMs (device query) x {FP32_LANES_PER_SM} FP32 FMA lanes x 2 flop x "
                    f"{mhz:.0f} MHz (sampled max SM clock)")
        traffic = None
        if dom in MEASURED_TRAFFIC:
            tb, grids = MEASURED_TRAFFIC[dom]
            traffic = tb * (3 * R) / grids
        roofline = {"bound": bound, "achieved": achieved, "peak": peak, "unit": u, "frac": achieved / peak,
                    "traffic": traffic, "kernel": dom, "peak_source": psrc,
                    "algorithmic_per_launch": amount, "algorithmic_unit": unit, "launch_ms": ms_dom / n_dom,
                    "timed_in": "stage-timed run of the same step (%d steps)" % Kp}
        sb = stage_bytes(dom, ctx)
        if sb:
            # the same launch on the HBM basis: unique bytes / launch time against the copy bandwidth
            roofline["hbm_basis"] = {"achieved": sb / sec / 1e9, "peak": hbm, "unit": "GB/s",
                                     "frac": sb / sec / 1e9 / hbm, "bytes_per_launch": sb,
                                     "peak_source": f"{src} copy bandwidth (MEASURED_PEAKS.json hbm_gbs)"}
        for s in stage_table:
            wk = stage_work(s, ctx)
            if wk:
                sec = stage_table[s]["ms_per_step"] * Kp / stage_table[s]["launch_groups"] / 1e3
                stage_table[s]["bound"] = wk[0]
                stage_table[s]["achieved"] = wk[1] / sec / (1e9 if wk[0] == "hbm" else 1e12)
                stage_table[s]["achieved_unit"] = "GB/s" if wk[0] == "hbm" else "TFLOP/s"

    # end to end through host buffers (pinned)
    xh = x.cpu().pin_memory()
    zh = torch.empty_like(xh).pin_memory()
    for _ in range(2):
        x.copy_(xh, non_blocking=True)
        step(PREC_MIXED)
        zh.copy_(z, non_blocking=True)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    Ke = max(3, K // 2)
    e0.record(stream)
    for _ in range(Ke):
        x.copy_(xh, non_blocking=True)
        step(PREC_MIXED)
        zh.copy_(z, non_blocking=True)
    e1.record(stream)
    torch.cuda.synchronize()
    e2e_val, _ = aggregate(e0.elapsed_time(e1) / 1e3, R * Ke, dist)
    e2e = {"value": e2e_val, "unit": "matvec/s", "h2d_bytes_per_step": int(xh.numel() * 16),
           "d2h_bytes_per_step": int(zh.numel() * 16)}

    # factorisation route of the preconditioner (band LDL^T or nested dissection)
    ndi = api.precond_nd_info(P)
    precond_route = ({"method": "nested dissection", "fronts": ndi["fronts"], "factor_entries": ndi["nnz"],
                      "max_front": ndi["max_front"], "complex_macs": ndi["flops"]}
                     if ndi["method"] == N.PC_ND else {"method": "band", **api.precond_info(P)})
    gm = None
    if not args.no_gmres:
        # residual: the preconditioned relative residual of the solve (FP64 for
        # plain_fp64; for the refined forms P^-1 (b - Z x) with an FP64 product
        # (mixed_refined) or a double-float one (mixed_refined_df), P^-1 and the
        # norms in FP64; the mixed operator's own for mixed)
        gm = {"tol": 1e-6, "rhs": R}
        for nm, prec, refine in (("plain_fp64", PREC_FP64, REFINE_OFF), ("mixed", PREC_MIXED, REFINE_OFF),
                                 ("mixed_refined", PREC_MIXED, REFINE_FP64),
                                 ("mixed_refined_df", PREC_MIXED, REFINE_DF)):
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            Z, st = api.sie_solve(P, freqs, tol=1e-6, restart=100, max_iter=400, prec=prec, refine=refine)
            dt = time.perf_counter() - t0
            gm[nm] = {"seconds": dt, "iterations_max": st["iterations_max"], "converged": st["converged"],
                      "residual_max": st["residual_max"], "matvecs": st["matvecs"]}
            if nm == "plain_fp64":
                Zref = Z
            else:
                gm[nm]["Z_rel_vs_plain"] = float(np.abs(Z - Zref).max() / np.abs(Zref).max())
        # the mixed solve converged on an FP64-class residual is the comparable one
        gm["headline"] = "mixed_refined_df"
        gm["speedup_vs_plain"] = gm["plain_fp64"]["seconds"] / gm["mixed_refined_df"]["seconds"]

    lossy = None
    if args.lossy and not args.graph:
        # the lossy-kernel variant on the same workload: per-frequency slots (complex spectrum
        # and near blocks) built on the first product, then the mixed step timed like the headline
        Pl = api.Plan(M, L, dict(PLAN_PARAMS, grid=w["grid"], kernel=N.KERNEL_LOSSY))
        yl, zl = torch.empty_like(x), torch.empty_like(x)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        api.pfft_matvec(Pl, x, om, SPACE_LOOP, PREC_MIXED, out=yl)
        t_slots = time.perf_counter() - t0

        def lstep():
            api.pfft_matvec(Pl, x, om, SPACE_LOOP, PREC_MIXED, out=yl)
            if args.step != "matvec":
                api.pfft_precond_apply(Pl, yl, om, out=zl, prec=PREC_MIXED)
        for _ in range(3):
            lstep()
        torch.cuda.synchronize()
        Kl = max(3, K // 3)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(Kl):
            lstep()
        e1.record(stream)
        torch.cuda.synchronize()
        tl = e0.elapsed_time(e1) / 1e3
        lossy = {"value": R * Kl / tl, "unit": "matvec/s", "ms_per_step": 1e3 * tl / Kl,
                 "kernel": "exp(-jkR)/R, k = (1 - j)/delta per right-hand side's frequency",
                 "first_product_seconds": t_slots, "frequencies": len(freqs),
                 "device_bytes": Pl.info()["device_bytes"]}
        del Pl

    pdn = None
    if args.plane_pair and world == 1 and args.workload == "bondwires_8x2mm_40k" and not args.graph:
        # the largest single-GPU configuration, in the same line; its failure must not
        # cost the headline, so it is reported instead of raised
        try:
            pdn = plane_pair_line(args.no_gmres)
        except Exception as e:  # noqa: BLE001
            pdn = {"workload": "pdn_2x10mm_500k", "error": f"{type(e).__name__}: {e}"}

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu:
        # one warm-up product builds the oracle's sparse near matrix (it is built lazily on the
        # first product), so the timed samples are products only, as in the reference arm
        rate, sample, _ = cpu_oracle_rate(args.workload, steps=5, warmup=1)
        cpu = {"value": rate, "unit": "matvec/s", "cores": os.cpu_count(), "kind": "oracle", "sample": sample}

    if rank == 0:
        line = {"metric": metric, "value": value, "unit": "matvec/s", "n_gpus": world, "steps": K, "warmup": W,
                "ms_per_step": 1e3 * tmax / K, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
                "dtype": "f32+f64", "data": "synthetic",
                "config": {"workload": w["name"], "triangles": int(m.nt), "loops": int(L.nl),
                           "grid": list(w["grid"]), "rhs_per_step": R, "frequencies": len(freqs), "ports": nports,
                           "near_pairs": info["n_near_pairs"],
                           "precond": precond_route,
                           "step": ("z = P^-1 A Z_b A^T x (mixed)" if args.step != "matvec" else "y = A Z_b A^T x (mixed)")
                           + (", replayed as a CUDA graph" if args.graph else ""),
                           "l2": "inputs larger than L2 (per-step grids %.2f GB, x-padded grids %.2f GB)" % (
                               3 * R * Nx * Ny * Nz * 8 / 1e9, 6 * R * Nx * Ny * Nz * 8 / 1e9),
                           "parallelism": f"replicas x{world}"},
                "plain_fp64": {"value": value_plain, "unit": "matvec/s", "ms_per_step": 1e3 * t_plain / max(3, K // 3)},
                "gmres": gm, "lossy_kernel": lossy, "plane_pair": pdn, "roofline": roofline,
                "stages": stage_table,
                "cpu_baseline": cpu, "e2e": e2e,
                "clocks": clocks, "gpu_launches": launches}
        print(json.dumps(line))
    if dist:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
