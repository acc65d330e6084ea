#!/usr/bin/env python
"""Throughput of the Hessian-preconditioned HMC hot path of arXiv:2504.07090 on one GB300.

One step = one HMC iteration on the 37-antenna HERA-like workload (cfg1: 64 channels
140-160 MHz, 60 LSTs, 128x192 pixels, 128x128 sky modes per channel + 4 complex gain
modes per antenna, 1,048,872 parameters): draw the momentum p = L z through the
preconditioner's Cholesky factor, then one 20-step leapfrog trajectory through
fm_leapfrog (21 chi^2+gradient evaluations: mode->pixel, beam, in-kernel fringe
phasors, tensor-core contraction, gains, chi^2, tensor-core adjoint, pixel->mode,
gain gradient, kicks, block-triangular drift, FP64 Hamiltonian, Metropolis test).

Prints one JSON line (rank 0).  value = chi^2+grad evaluations/s of the whole job.
`--impl reference` times the FP64 CPU oracle instead (bounded samples, host cores).
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
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "χ²+grad evals/s & vis-pixel terms/s at stated err vs FP64; leapfrog steps/s"
FALLBACK_PEAKS = {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "bf16_tflops_sustained": 1700.0}
N_PRODUCTS = {"bf16x1": 1, "fp16x1": 1, "bf16x3": 3, "fp16x3": 3}
# leapfrog step per workload: the largest with acceptance above 90 % (Sec. 4.2); at cfg1 the
# energy error of a 20-step trajectory grows as eps^4 (median |dH| 0.43 at 0.01, 7.4 at 0.02)
EPS_DEFAULT = {"cfg1": 0.007, "cfg3": 0.007, "cfg4": 0.004}
A_MIN = 0.2                 # acceptance threshold of the step-size rule (App. B)
LEGENDRE_ORDERS = 6          # cfg1 compressed: 64 channels onto 6 Legendre orders (98,600 parameters)
# DRAM read + write bytes per launch of the dominant kernel (dram__bytes_read.sum +
# dram__bytes_write.sum), from the ncu capture of profiles/k_vis_ha_k_adj_ha_cfg1_fp16x3.md,
# keyed (workload, precision, form, kernel); a kernel changed since its capture has no entry
# (the forward's capture, 305.163264e6 + 4.400384e6 bytes, was taken with 16 producer warps: its
# entry is left out since the kernel runs 12)
TRAFFIC = {("cfg1", "fp16x3", "hour_angle", "adj"): 296.406272e6 + 7.381760e6}


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--config", default="cfg1")
    ap.add_argument("--precision", default=None, help="default: fp16x3 (cfg1), bf16x3 (cfg2)")
    ap.add_argument("--problems", type=int, default=64, help="cfg2: number of independent problems")
    ap.add_argument("--traj", type=int, default=20, help="leapfrog steps per trajectory")
    ap.add_argument("--eps", type=float, default=None, help="leapfrog step: default 0.007 (cfg1), 0.02 (cfg2)")
    ap.add_argument("--block", type=int, default=64, help="preconditioner block (64, or 1 for the diagonal)")
    ap.add_argument("--no-forms", action="store_true", help="skip the bf16x3 / fp32 comparison and the errors")
    ap.add_argument("--no-err", action="store_true", help="skip the errors against the FP64 oracle")
    ap.add_argument("--cpu-seconds", type=float, default=12.0, help="budget of the oracle timing sample")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cfg4", action="store_true", help="cfg1: skip the cfg4 measurement in the same line")
    ap.add_argument("--no-cfg3", action="store_true", help="cfg1: skip the preconditioner / HVP measurement")
    ap.add_argument("--no-cfg2", action="store_true", help="cfg1: skip the batched uneven-problem measurement")
    ap.add_argument("--no-legendre", action="store_true",
                    help="cfg1: skip the measurement with the sky compressed onto Legendre orders in frequency")
    ap.add_argument("--no-tune", action="store_true", help="cfg2: keep the default launch grids")
    ap.add_argument("--hvps", type=int, default=1000, help="cfg3: Gauss-Newton HVPs timed")
    return ap.parse_args()


def peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as fh:
            d = json.load(fh)
        return {k: float(d[k]) for k in FALLBACK_PEAKS}, "measured"
    except Exception:
        return dict(FALLBACK_PEAKS), "fallback"


def workload_desc(prob, traj, block=64):
    pc = "64-block" if block > 1 else "diagonal"
    return (f"{prob.name}: {prob.n_ant}-antenna hexagon ({prob.n_bl} baselines), {prob.n_freq} ch "
            f"{prob.freq_hz[0] / 1e6:.0f}-{prob.freq_hz[-1] / 1e6:.0f} MHz, {prob.n_lst} LSTs, "
            f"{prob.n_dec}x{prob.n_ra} px, {prob.n_mode_ra}x{prob.n_mode_dec} modes/"
            f"{'ch' if not prob.n_freq_modes else f'Legendre order ({prob.n_freq_modes} orders in frequency)'}, "
            f"{prob.n_params} params; one HMC iteration = p = L z + {traj}-step leapfrog ({traj + 1} chi2+grad evals), "
            f"{pc} Gauss-Newton mass matrix")


# ------------------------------------------------------------------ ranks
def job_rate(local_ms: float, units_per_rank: float, world: int, dist=None, device=None):
    """Whole-job rate over `world` ranks that each process units_per_rank units: the job's time
    is the slowest rank's (an all-reduce MAX of local_ms when dist is given).  Returns
    (units per second of the whole job, that time in ms)."""
    ms = float(local_ms)
    if dist is not None:
        import torch
        t = torch.tensor([ms], dtype=torch.float64, device=device)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        ms = float(t.item())
    return world * units_per_rank / (ms / 1000.0), ms


# ------------------------------------------------------------------ clocks
class ClockSampler:
    """nvidia-smi samples every 50 ms, started before the warm-up; stop() keeps the samples
    whose own timestamps fall inside the window marked by begin() / end() (all samples,
    and "window": "run", when none do, e.g. for a window shorter than the interval, or when
    nvidia-smi does not take the timestamp field and is restarted without it)."""
    QUERY = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
    NAMES = ("hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap")

    def __init__(self, gpu_index: int):
        self.path = tempfile.mktemp(suffix=".csv")
        self.proc = None
        self.gpu = gpu_index
        self.stamped = True
        self.t0 = self.t1 = None

    def _launch(self, fields: str) -> bool:
        """Start nvidia-smi; True once it has written a sample (waits up to 3 s)."""
        self.fh = open(self.path, "w")
        self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.gpu}", f"--query-gpu={fields}",
                                      "--format=csv,noheader,nounits", "-lms", "50"],
                                     stdout=self.fh, stderr=subprocess.DEVNULL)
        deadline = time.time() + 3.0
        while time.time() < deadline:
            if os.path.getsize(self.path) > 0:
                return True
            if self.proc.poll() is not None:
                break
            time.sleep(0.02)
        return os.path.getsize(self.path) > 0

    def start(self):
        try:
            if not self._launch("timestamp,index," + self.QUERY) and self.proc.poll() is not None:
                self.fh.close()
                self.stamped = False
                self._launch("index," + self.QUERY)
        except Exception:
            self.proc = None

    def begin(self):
        self.t0 = time.time()

    def end(self):
        self.t1 = time.time()

    @staticmethod
    def parse(lines, t0=None, t1=None, stamped=True, slack=0.06):
        """Samples of nvidia-smi csv lines ([timestamp,] index, then QUERY); with t0 / t1
        (epoch seconds) only those stamped within [t0 - slack, t1 + slack], if any."""
        import datetime
        off = 1 if stamped else 0
        rows = []
        for line in lines:
            parts = [x.strip() for x in line.split(",")]
            if len(parts) < 9 + off:
                continue
            try:
                sm, smax = float(parts[1 + off]), float(parts[2 + off])
            except ValueError:
                continue
            ts = None
            if stamped:
                try:
                    ts = datetime.datetime.strptime(parts[0], "%Y/%m/%d %H:%M:%S.%f").timestamp()
                except ValueError:
                    ts = None
            flags = parts[5 + off:9 + off]
            act = {nm for nm, v in zip(ClockSampler.NAMES, flags) if v.lower().startswith("active")}
            rows.append((ts, sm, smax, act))
        window = "run"
        if t0 is not None and t1 is not None:
            inside = [r for r in rows if r[0] is not None and t0 - slack <= r[0] <= t1 + slack]
            if inside:
                rows, window = inside, "timed region"
        sm = [r[1] for r in rows]
        reasons = set().union(*[r[3] for r in rows]) if rows else set()
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(r[2] for r in rows) if rows else None,
                "samples": len(sm), "window": window, "reasons": sorted(reasons)}

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.fh.close()
        with open(self.path) as fh:
            out = self.parse(fh.readlines(), self.t0, self.t1, self.stamped)
        os.unlink(self.path)
        return out


# ------------------------------------------------------------------ CPU oracle
def oracle_sample_rate(prob, theta, d, budget_s: float):
    """chi^2+grad evals/s of the FP64 oracle, from a bounded sample: the pixel<->mode
    transforms of one channel and the fringe sum + adjoint of k (channel, LST) pairs,
    extrapolated linearly to all channels and pairs (the work is exactly linear in both)."""
    import oracle
    o = oracle.Oracle(prob)
    o.sigma = prob.sigma
    a, gam = o.split(theta)
    t0 = time.perf_counter()
    x0 = o.sky_f(a[0])
    abar = o.sky_adjoint_f(x0)
    t_chan = time.perf_counter() - t0
    g = o.gains(gam)
    k, t_pairs = 0, 0.0
    while True:
        t = k % prob.n_lst
        t1 = time.perf_counter()
        V = o.vis_ft(0, t, x0)
        r = g[0, o.bl_i] * np.conj(g[0, o.bl_j]) * V - d[0, t]
        omega = np.conj(g[0, o.bl_i]) * g[0, o.bl_j] * r / o.sigma ** 2
        xbar = np.zeros(o.npix)
        o.adjoint_ft(0, t, omega, xbar)
        t_pairs += time.perf_counter() - t1
        k += 1
        if t_pairs + t_chan > budget_s or k >= prob.n_lst:
            break
    per_eval = prob.n_freq * t_chan + prob.n_freq * prob.n_lst * (t_pairs / k)
    sample = (f"1 channel of pixel<->mode transforms ({t_chan:.2f} s) + {k} (channel, LST) pairs of fringe sum "
              f"and adjoint ({t_pairs:.2f} s), extrapolated to {prob.n_freq} channels x {prob.n_lst} LSTs")
    return 1.0 / per_eval, oracle.num_threads(), sample, t_chan + t_pairs


def run_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    from paper_2504_07090_gb300 import synth
    prob = synth.config(args.config)
    tr = synth.draw_truth(prob)
    rng = np.random.default_rng(1)
    prob.sigma = 1.0
    d = rng.standard_normal((prob.n_freq, prob.n_lst, prob.n_bl)) * 10 + 0j
    budget = max(1.0, min(args.cpu_seconds, 120.0 / max(1, args.steps + args.warmup)))
    rates = []
    cores = 1
    sample = ""
    for i in range(args.warmup + args.steps):
        r, cores, sample, _ = oracle_sample_rate(prob, tr.theta, d, budget)
        if i >= args.warmup:
            rates.append(r)
    v = float(np.mean(rates))
    print(json.dumps({
        "impl": "reference", "metric": METRIC, "value": v, "unit": "chi2+grad evals/s",
        "n_gpus": int(os.environ.get("WORLD_SIZE", str(args.gpus))),         # the launch's N (host cores)
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1000.0 / v, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": workload_desc(prob, args.traj)},      # the GPU arm's workload and unit
        "cpu_baseline": {"value": v, "unit": "chi2+grad evals/s", "cores": cores, "kind": "oracle", "sample": sample},
        "e2e": {"value": v, "unit": "chi2+grad evals/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
        "note": "the FP64 oracle timed on a bounded sample of every step and extrapolated linearly to the whole "
                "evaluation (the work is linear in channels and (channel, LST) pairs), so ms_per_step x steps is "
                "far longer than this run's wall clock by design",
    }), flush=True)


# ------------------------------------------------------------------ GPU arm
def main_batch(args):
    """cfg2 alone (`--config cfg2`): one JSON line."""
    import torch
    from paper_2504_07090_gb300 import build
    if int(os.environ.get("RANK", "0")) != 0:
        return
    torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", "0")))
    build.build()
    line = measure_batch(args, args.steps, args.warmup)
    print(json.dumps(line), flush=True)


def measure_batch(args, K, W):
    """cfg2: independent HMC chains on problems of uneven size (antennas 7/19/37, 16/32/64
    channels, 512..16384 modes per channel, 20 LSTs).  One step = for every chain p = L z,
    then one launch of the CUDA graph holding every chain's trajectory (fm_batch_leapfrog)."""
    import torch
    from paper_2504_07090_gb300 import fm, synth
    prec = args.precision or "bf16x3"
    probs = synth.batch_problems(args.problems)
    dev = "cuda"
    t_setup = time.perf_counter()
    models, qs, ps, zs, forms = [], [], [], [], {}
    for k, prob in enumerate(probs):
        tr = synth.draw_truth(prob)
        h0 = fm.ForwardModel(prob, prec, sigma=1.0)
        th = torch.tensor(tr.theta, dtype=torch.float32, device=dev)
        m = h0.forward(th)
        sigma = 0.01 * float(torch.linalg.norm(m, dim=-1).mean())
        h0.close()
        prob.sigma = sigma
        h = fm.ForwardModel(prob, prec, sigma=sigma)
        h.set_data((m + sigma * torch.tensor(tr.noise, dtype=torch.float32, device=dev)).contiguous())
        mu, lam = synth.prior_for(prob, tr.theta)
        h.set_prior(torch.tensor(mu, dtype=torch.float32, device=dev), torch.tensor(lam, dtype=torch.float32, device=dev))
        nk = prob.n_mode_ra * prob.n_mode_dec
        h.build_precond(th, 64 if nk % 64 == 0 else 1)
        models.append(h)
        qs.append(th.clone())
        ps.append(torch.empty_like(th))
        zs.append(torch.tensor(synth.random_vectors(h.n_params, K + W, 20250430 + k), dtype=torch.float32, device=dev))
        f = h.contraction_info()["form"]
        forms[f] = forms.get(f, 0) + 1
    torch.cuda.synchronize()
    t_setup = time.perf_counter() - t_setup
    n = len(models)
    # launch grids per problem from the autotuner (timings cached by problem shape)
    eps = [args.eps or min(0.03, 0.007 * (1048872.0 / h.n_params) ** 0.25) for h in models]
    tune = None
    if not args.no_tune:
        from paper_2504_07090_gb300 import autotune
        st0 = torch.cuda.current_stream()

        def run_step():
            b = fm.Batch(models, qs, ps, args.traj)
            u0 = [0.5] * n
            for k in range(n):
                models[k].precond_apply(0, zs[k][0], out=ps[k])
            b.run(eps, u0)
            torch.cuda.synchronize()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(st0)
            for _ in range(2):
                for k in range(n):
                    models[k].precond_apply(0, zs[k][0], out=ps[k])
                b.run(eps, u0)
            e1.record(st0)
            torch.cuda.synchronize()
            b.close()
            return e0.elapsed_time(e1) / 2

        tune = autotune.tune_batch(models, qs, run_step)
    batch = fm.Batch(models, qs, ps, args.traj)
    # step per chain (set above): cfg1's 0.007 scaled by the parameter count to the power -1/4
    # (the energy error of a trajectory grows as n_params eps^4), at most 0.03
    us = np.random.default_rng(20250431).random((K + W, n))
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)
    st = torch.cuda.current_stream()

    def draw(i):
        for k in range(n):
            models[k].precond_apply(0, zs[k][i], out=ps[k])

    clocks = ClockSampler(int(os.environ.get("LOCAL_RANK", "0")))
    clocks.start()
    for i in range(W):
        flush.zero_()
        draw(i)
        batch.run(eps, us[i])
    torch.cuda.synchronize()
    for h in models:
        h.sync_status()
    l0 = fm.kernel_launches()
    evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(K)]
    clocks.begin()
    for i in range(K):
        flush.zero_()
        evs[i][0].record(st)
        draw(W + i)
        batch.run(eps, us[W + i])
        evs[i][1].record(st)
    torch.cuda.synchronize()
    clocks.end()
    clk = clocks.stop()
    launches = fm.kernel_launches() - l0 + K * batch.kernels()
    acc_last = int(sum(int(a.item()) for a in batch.acc_out))
    for h in models:
        h.sync_status()
    total_ms = float(sum(a.elapsed_time(b) for a, b in evs))
    # the same trajectories launched one chain after another (fm_leapfrog, no graph)
    seq_ms = 0.0
    for i in range(min(K, 2)):
        flush.zero_()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(st)
        draw(W + i)
        for k in range(n):
            models[k].leapfrog(qs[k], ps[k], eps[k], args.traj, float(us[W + i][k]), batch.h_out[k], batch.acc_out[k])
        b.record(st)
        torch.cuda.synchronize()
        seq_ms += a.elapsed_time(b)
    seq_ms /= min(K, 2)
    evals = n * (args.traj + 1)
    value = K * evals / (total_ms / 1000.0)
    n_par = sum(h.n_params for h in models)
    line = {
        "metric": METRIC, "value": value, "unit": "chi2+grad evals/s", "n_gpus": 1, "steps": K, "warmup": W,
        "ms_per_step": total_ms / K, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "f32", "precision": prec, "data": "synthetic",
        "config": {"workload": f"cfg2: {n} independent problems (antennas 7/19/37, 16/32/64 channels, 20 LSTs, "
                               f"512..16384 modes per channel; {n_par} parameters in all; contraction forms {forms}); "
                               f"one step = p = L z per chain + one graph launch of {n} {args.traj}-step trajectories "
                               f"({evals} chi2+grad evals)",
                   "l2": "flushed between steps (256 MB write)", "parallelism": "single GPU, concurrent graph branches"},
        "leapfrog_steps_per_s": K * n * args.traj / (total_ms / 1000.0),
        "sequential_launch_ms_per_step": seq_ms, "setup_s": t_setup, "autotune": tune,
        "sampler": {"eps": {"min": min(eps), "max": max(eps)}, "n_steps": args.traj,
                    "accepted_in_last_step": acc_last, "chains": n},
        "roofline": None, "cpu_baseline": None, "e2e": None, "gpu_launches": int(launches), "clocks": clk,
    }
    batch.close()
    for h in models:
        h.close()
    return line


def errors_vs_fp64(prob, tr, handles, d_dev, f0):
    """Relative l2 errors of the GPU forms against the FP64 oracle on channel f0 of the timed
    workload: the visibilities of all its LSTs at the truth, and its sky gradient at sky modes
    perturbed by 1 % of the channel rms.  For the gradient each handle gets, for the duration
    of the check, data that are the oracle model plus seeded noise on channel f0 and zero on
    the others (the sky modes are per channel, so that slice of the gradient depends on f0
    alone); the oracle's restricted gradient plus the prior's is the expected value."""
    import torch
    import oracle
    o = oracle.Oracle(prob)
    o.sigma = prob.sigma
    th = tr.theta.astype(np.float32).astype(np.float64)
    t0 = time.perf_counter()
    pairs = [(f0, t) for t in range(prob.n_lst)]
    m0 = o.model(th, fts=pairs)[f0]
    a, _ = o.split(th)
    sc = np.zeros(o.n_par)
    sc[: o.n_sky] = np.repeat(np.sqrt(np.mean(a ** 2, axis=1)), o.nk)
    th_e = (th + 0.01 * sc * np.random.default_rng(6).standard_normal(o.n_par)).astype(np.float32).astype(np.float64)
    d1 = np.zeros((prob.n_freq, prob.n_lst, prob.n_bl, 2))
    d1[f0] = np.stack([m0.real, m0.imag], -1) + prob.sigma * tr.noise[f0]
    d1 = d1.astype(np.float32).astype(np.float64)
    _, _, g = o.chi2_grad(th_e, d1[..., 0] + 1j * d1[..., 1], fts=pairs)
    from paper_2504_07090_gb300 import synth
    mu, lam = synth.prior_for(prob, tr.theta)
    sl = slice(f0 * o.nk, (f0 + 1) * o.nk)
    g_sl = g[sl] + (lam * (th_e - mu.astype(np.float32).astype(np.float64)))[sl]
    t_or = time.perf_counter() - t0
    out = {}
    d1_dev = torch.tensor(d1, dtype=torch.float32, device="cuda").contiguous()
    for name, h in handles.items():
        V = h.forward(torch.tensor(th, dtype=torch.float32, device="cuda"))[f0].double().cpu().numpy()
        ev = float(np.linalg.norm(V[..., 0] + 1j * V[..., 1] - m0) / np.linalg.norm(m0))
        h.set_data(d1_dev)
        _, grad = h.chi2_grad(torch.tensor(th_e, dtype=torch.float32, device="cuda"))
        eg = float(np.linalg.norm(grad[sl].double().cpu().numpy() - g_sl) / np.linalg.norm(g_sl))
        h.set_data(d_dev)
        out[name] = {"V": ev, "grad": eg}
    return out, {"channel": int(f0), "pairs": len(pairs), "oracle_s": t_or,
                 "what": f"relative l2 vs the FP64 oracle: all {prob.n_lst}x{prob.n_bl} visibilities of channel {f0} "
                         f"at the truth; its {o.nk} sky-gradient entries at a 1 % sky perturbation"}


def errors_sampled(prob, tr, h, n):
    """Relative l2 error of n visibilities at the truth, sampled over channels, LSTs (both
    halves of the LST range) and baselines, each computed one by one by the FP64 oracle."""
    import torch
    import oracle
    o = oracle.Oracle(prob)
    th = tr.theta.astype(np.float32).astype(np.float64)
    a, gam = o.split(th)
    g = o.gains(gam)
    rng = np.random.default_rng(4)
    t0 = time.perf_counter()
    fs = rng.choice(prob.n_freq, 4, replace=False)
    idx, want = [], []
    for f in fs:
        x_f = o.sky_f(a[f])
        for k in range(n // 4):
            t = int(rng.integers(prob.n_lst // 2)) + (prob.n_lst // 2 if k % 2 else 0)
            b = int(rng.integers(prob.n_bl))
            idx.append((int(f), t, b))
            want.append(o.vis_one(int(f), t, b, x_f) * g[f, o.bl_i[b]] * np.conj(g[f, o.bl_j[b]]))
    V = h.forward(torch.tensor(th, dtype=torch.float32, device="cuda"))
    ii = torch.tensor(idx, dtype=torch.long, device="cuda")
    got = V[ii[:, 0], ii[:, 1], ii[:, 2]].double().cpu().numpy()
    got = got[:, 0] + 1j * got[:, 1]
    want = np.array(want)
    return {"V": float(np.linalg.norm(got - want) / np.linalg.norm(want)), "grad": None,
            "samples": len(idx), "oracle_s": time.perf_counter() - t0,
            "what": f"relative l2 vs the FP64 oracle of {len(idx)} visibilities at the truth (4 channels, LSTs from "
                    "both passes, random baselines), each summed one by one; the gradient is not compared at this "
                    "size (the oracle takes minutes per channel)"}


def measure_cfg3(h, q, prob, flush, st, n_hvp):
    """cfg3 on the cfg1 handle: the Gauss-Newton mass-matrix builds (diagonal and 64-blocks,
    FP64 accumulation) and n_hvp Hessian-vector products with N(0, 1) vectors drawn on the
    device (Philox), CUDA events around the loop; the HVP's error is checked against central
    differences of the device gradient along sky-only vectors (exact: U is quadratic there)."""
    import torch
    from paper_2504_07090_gb300 import fm
    out = {"workload": "cfg3: cfg1 sizes (1048872 parameters); diagonal and 64 x 64 block Gauss-Newton builds, "
                       f"{n_hvp} HVPs with N(0,1) vectors"}
    for bs in (1, 64):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        h.build_precond(q, bs)
        torch.cuda.synchronize()
        out[f"build_s_block{bs}"] = time.perf_counter() - t0
    hv = torch.empty_like(q)
    for full in (False, True):
        n = n_hvp if not full else max(1, n_hvp // 10)
        vs = [fm.draw_normal(777, k, h.n_params) for k in range(4)]
        h.hvp(q, vs[0], full=full, out=hv)
        flush.zero_()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(st)
        for k in range(n):
            v = fm.draw_normal(777, k, h.n_params) if k < 4 else vs[k % 4]
            h.hvp(q, v, full=full, out=hv)
        b.record(st)
        torch.cuda.synchronize()
        ms = a.elapsed_time(b)
        out["gn" if not full else "full"] = {"hvps": n, "hvp_per_s": n / (ms / 1000.0), "ms_per_hvp": ms / n,
                                             "note": "each iteration also draws its N(0,1) vector on the device"}
    # full Hessian along sky-only vectors against central differences of the gradient
    n_sky = prob.n_sky_params
    errs = []
    g1, g2 = torch.empty_like(q), torch.empty_like(q)
    for k in range(3):
        v = fm.draw_normal(991, k, h.n_params)
        v[n_sky:] = 0.0
        v /= torch.linalg.norm(v)
        hvk = h.hvp(q, v, full=True).double()
        h.chi2_grad(q, g1)
        # a step whose gradient change is as large as the gradient itself (FP32 gradients)
        step = float(torch.linalg.norm(g1.double())) / float(torch.linalg.norm(hvk))
        h.chi2_grad(q + step * v, g1)
        h.chi2_grad(q - step * v, g2)
        fd = (g1.double() - g2.double()) / (2.0 * step)
        errs.append(float(torch.linalg.norm(fd - hvk) / torch.linalg.norm(fd)))
    out["hvp_vs_gradient_differences"] = {"max_rel_l2": max(errs), "vectors": 3,
                                          "what": "full HVP along sky-only unit vectors vs central differences of "
                                                  "the device gradient (exact for any step: U is quadratic in the sky)"}
    return out


def time_chi2_grad(h, theta, n_eval, reps, flush, st):
    """chi^2 + gradient evaluations/s of one handle: reps x n_eval back-to-back fm_chi2_grad
    calls, L2 flushed before each batch, CUDA events around each batch."""
    import torch
    scal = torch.empty(2, dtype=torch.float64, device="cuda")
    grad = torch.empty_like(theta)
    h.chi2_grad(theta, grad, scal)
    tot = 0.0
    for _ in range(reps):
        flush.zero_()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(st)
        for _ in range(n_eval):
            h.chi2_grad(theta, grad, scal)
        b.record(st)
        torch.cuda.synchronize()
        tot += a.elapsed_time(b)
    return reps * n_eval / (tot / 1000.0), tot / (reps * n_eval)


def measure(args, name, K, W, rank, world, dist, local, forms_on=True, err_mode="channel", freq_modes=0):
    """One workload end to end: handle, mock data, prior and mass matrix; W warm-up and K timed
    HMC iterations (fm_hmc_chain, one graph launch each, L2 flushed between them); the kernel
    split from a profiled pass; e2e through host buffers; the other forms and the errors
    against the FP64 oracle (err_mode "channel": one channel's visibilities and sky gradient,
    "sampled": visibilities one by one); the oracle's CPU rate.  freq_modes > 0 compresses the
    sky onto that many Legendre orders in frequency.  Returns the line's fields."""
    import torch
    from paper_2504_07090_gb300 import fm, synth
    prob = synth.config(name)
    if freq_modes:
        prob = synth.with_freq_modes(prob, freq_modes)
    tr = synth.draw_truth(prob)
    dev = "cuda"
    # mock data: model at the truth plus noise of 1 % of the mean |V| per real component
    h0 = fm.ForwardModel(prob, args.precision, sigma=1.0)
    th_true = torch.tensor(tr.theta, dtype=torch.float32, device=dev)
    m = h0.forward(th_true)
    sigma = 0.01 * float(torch.linalg.norm(m, dim=-1).mean())
    h0.close()
    prob.sigma = sigma
    h = fm.ForwardModel(prob, args.precision, sigma=sigma)
    d = (m + sigma * torch.tensor(tr.noise, dtype=torch.float32, device=dev)).contiguous()
    del m
    h.set_data(d)
    mu, lam = synth.prior_for(prob, tr.theta)
    mu_d = torch.tensor(mu, dtype=torch.float32, device=dev)
    lam_d = torch.tensor(lam, dtype=torch.float32, device=dev)
    h.set_prior(mu_d, lam_d)
    q = th_true.clone()
    t_pc = time.perf_counter()
    h.build_precond(q, args.block)
    torch.cuda.synchronize()
    t_pc = time.perf_counter() - t_pc

    # the chain runs on the device (fm_hmc_chain): momentum z ~ N(0, 1) from the counter-based
    # generator, p = L z, the trajectory, the Metropolis test and the step-size rule of App. B,
    # one captured graph launch per HMC iteration
    seed = 20250420 + rank
    state = torch.tensor([args.eps, 0.0], dtype=torch.float64, device=dev)
    trace = torch.zeros((W + K, 5), dtype=torch.float64, device=dev)
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)   # > L2 (126 MB)
    st = torch.cuda.current_stream()

    def step(i):
        h.hmc_chain(q, 1, args.traj, args.eps, A_MIN, seed, state, trace[i])

    clocks = ClockSampler(local)
    clocks.start()
    for i in range(W):
        flush.zero_()
        step(i)
    torch.cuda.synchronize()
    h.sync_status()

    # ---- timed region: profiling off
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    clocks.begin()
    launches0 = fm.kernel_launches()
    evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(K)]
    torch.cuda.nvtx.range_push("bench_timed")
    for i in range(K):
        flush.zero_()
        evs[i][0].record(st)
        step(W + i)
        evs[i][1].record(st)
    torch.cuda.synchronize()
    clocks.end()
    torch.cuda.nvtx.range_pop()
    # kernels of the library in the timed region: one graph per iteration (fm_kernel_launches
    # counts launches made outside graphs, here the chain's call-setup kernel)
    launches = fm.kernel_launches() - launches0 + K * h.chain_kernels()
    clk = clocks.stop()
    if dist:
        dist.barrier()
    h.sync_status()
    step_ms = [a.elapsed_time(b) for a, b in evs]
    total_ms = float(sum(step_ms))
    evals_per_step = args.traj + 1
    value, total_ms = job_rate(total_ms, K * evals_per_step, world, dist, dev)
    rec = trace.cpu().numpy()[W:]
    dH = rec[:, 2] - rec[:, 1]
    sampler = {"eps0": args.eps, "a_min": A_MIN, "n_steps": args.traj, "trajectories": K,
               "accepted": int(rec[:, 3].sum()), "acceptance_rate": float(rec[:, 3].mean()),
               "mean_accept_prob": float(rec[:, 4].mean()), "median_abs_dH": float(np.median(np.abs(dH))),
               "eps_used": {"min": float(rec[:, 0].min()), "max": float(rec[:, 0].max())},
               "eps_after": float(state[0].item()),
               "rule": "Philox4x32-10 momentum and accept draws on the device; eps <- eps/1.2 if a < a_min else "
                       "min(eps0, 1.2 eps) (App. B); eps0 the largest step with acceptance above 90 % (Sec. 4.2)"}

    # ---- roofline of the dominant contraction kernel: a separate, untimed pass with the
    # per-launch events on (fm_set_profiling), over the same kind of steps
    h.get_profile()
    h.set_profiling(True)
    q_keep, state_keep = q.clone(), state.clone()
    p = torch.empty_like(q)
    hp = torch.empty(2, dtype=torch.float64, device=dev)
    ap = torch.empty(1, dtype=torch.int32, device=dev)
    zp = torch.tensor(synth.random_vectors(h.n_params, 1, seed)[0], dtype=torch.float32, device=dev)
    for i in range(min(K, 5)):
        # the same trajectories launched directly (fm_leapfrog), so that the events record
        flush.zero_()
        h.precond_apply(0, zp, out=p)
        h.leapfrog(q, p, args.eps, args.traj, 0.5, hp, ap)
    (fwd_ms, adj_ms), (fwd_n, adj_n) = h.get_profile()
    h.set_profiling(False)
    q.copy_(q_keep)
    state.copy_(state_keep)
    info = h.contraction_info()
    pk, pk_src = peaks()
    nprod = N_PRODUCTS.get(args.precision, 1)
    peak = pk["bf16_tflops_sustained"] / nprod
    fwd_ms1, adj_ms1 = fwd_ms / max(fwd_n, 1), adj_ms / max(adj_n, 1)
    if info["form"] == "hour_angle":
        # grouped complex-by-real contraction over the band of non-zero Toeplitz entries:
        # 4 flops per (fringe group, pixel, channel, LST), the same count for the adjoint
        flops_launch = 4.0 * info["fringes"] * prob.n_pix * prob.n_freq * prob.n_lst
        formula = "4 n_groups n_pix n_freq n_lst"
        names = ("forward contraction (k_vis_ha)", "adjoint contraction (k_adj_ha)")
        npad = (min(prob.n_lst, 64) + 15) // 16 * 16
        n_pass = (prob.n_lst + 63) // 64
        nhp = info["hour_angle_cells"]
        n_mt, n_kq = (info["fringes"] + 63) // 64, (info["fringes"] + 31) // 32
        exe = (n_pass * nprod * 2.0 * 128 * n_mt * npad * nhp * prob.n_dec * prob.n_freq,
               n_pass * nprod * 2.0 * nhp * npad * 64 * n_kq * prob.n_dec * prob.n_freq)
    else:
        flops_launch = 8.0 * prob.n_ant ** 2 * prob.n_pix * prob.n_freq * prob.n_lst
        formula = "8 n_ant^2 n_pix n_freq n_lst"
        names = ("forward contraction (k_vis_tc)", "adjoint contraction (k_adj_tc)")
        exe = (None, None)
    fwd_dom = fwd_ms >= adj_ms
    dom = names[0] if fwd_dom else names[1]
    dom_ms1, dom_n = (fwd_ms1, fwd_n) if fwd_dom else (adj_ms1, adj_n)
    achieved = flops_launch / (dom_ms1 / 1000.0) / 1e12 if dom_n else None
    traffic = TRAFFIC.get((name, args.precision, info["form"], "fwd" if fwd_dom else "adj"))
    roofline = {"bound": "tensor", "kernel": dom, "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
                "frac": achieved / peak if achieved else None, "traffic": traffic,
                "peak_source": f"{pk_src} bf16 sustained {pk['bf16_tflops_sustained']} TFLOP/s / {nprod} products "
                               f"(FP32-equivalent rate of the {args.precision} split); algorithmic flops per launch "
                               f"= {formula} = {flops_launch:.4g}",
                "form": info["form"], "fringes": info["fringes"],
                "forward_ms_per_launch": fwd_ms1, "adjoint_ms_per_launch": adj_ms1,
                "launches": {"forward": fwd_n, "adjoint": adj_n},
                "timing": "CUDA events around every contraction launch on its stream, in an untimed pass of "
                          f"{min(K, 5)} steps after the timed region"}
    if exe[0] is not None and dom_n:
        e_dom = exe[0] if fwd_dom else exe[1]
        roofline["tensor_executed_tflops"] = e_dom / (dom_ms1 / 1000.0) / 1e12
        roofline["tensor_executed_frac_of_bf16_sustained"] = roofline["tensor_executed_tflops"] / pk["bf16_tflops_sustained"]

    # ---- end to end through the C ABI with host buffers: H2D (q, z) -> step -> D2H (q, H, accepted)
    e2e = None
    if not args.no_e2e:
        qh = q.detach().cpu().pin_memory()
        q_back = torch.empty_like(qh).pin_memory()
        rec_h = torch.empty(5, dtype=torch.float64).pin_memory()
        torch.cuda.synchronize()
        e_ms = 0.0
        for i in range(K):
            flush.zero_()
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(st)
            q.copy_(qh, non_blocking=True)
            h.hmc_chain(q, 1, args.traj, args.eps, A_MIN, seed, state, trace[W + i])
            q_back.copy_(q, non_blocking=True)
            rec_h.copy_(trace[W + i], non_blocking=True)
            b.record(st)
            torch.cuda.synchronize()
            e_ms += a.elapsed_time(b)
        e_rate, e_ms = job_rate(e_ms, K * evals_per_step, world, dist, dev)
        e2e = {"value": e_rate, "unit": "chi2+grad evals/s",
               "h2d_bytes_per_step": 4 * h.n_params, "d2h_bytes_per_step": 4 * h.n_params + 5 * 8}

    # ---- the other forms on the same workload (chi^2 + gradient alone) and every form's
    # error against the FP64 oracle
    forms, err, err_info = None, None, None
    if rank == 0 and err_mode == "sampled" and not args.no_err:
        err = errors_sampled(prob, tr, h, 32)
    if rank == 0 and forms_on and not args.no_forms:
        q.copy_(th_true)
        handles = {args.precision: h}
        for pr in [x for x in ("fp16x3", "bf16x3", "fp32") if x != args.precision]:
            hx = fm.ForwardModel(prob, pr, sigma=sigma)
            hx.set_data(d)
            hx.set_prior(mu_d, lam_d)
            handles[pr] = hx
        forms = {}
        for pr, hx in handles.items():
            n_eval = evals_per_step if pr != "fp32" else 3
            rate, ms = time_chi2_grad(hx, q, n_eval, 3, flush, st)
            forms[pr] = {"chi2_grad_evals_per_s": rate, "ms_per_eval": ms, "form": hx.contraction_info()["form"]}
        if not args.no_err:
            f0 = int(np.random.default_rng(3).integers(prob.n_freq))
            err_all, err_info = errors_vs_fp64(prob, tr, handles, d, f0)
            for pr in forms:
                forms[pr]["err_vs_fp64"] = err_all[pr]
            err = dict(err_all[args.precision], **err_info)
        for pr, hx in handles.items():
            if hx is not h:
                hx.close()

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        dn = d.double().cpu().numpy()
        r, cores, sample, _ = oracle_sample_rate(prob, tr.theta, dn[..., 0] + 1j * dn[..., 1], args.cpu_seconds)
        cpu = {"value": r, "unit": "chi2+grad evals/s", "cores": cores, "kind": "oracle", "sample": sample}

    cfg3 = None
    if rank == 0 and name == "cfg1" and not freq_modes and not args.no_cfg3:
        q.copy_(th_true)
        cfg3 = measure_cfg3(h, q, prob, flush, st, args.hvps)
    out = {"value": value, "ms_per_step": total_ms / K, "steps": K, "warmup": W, "precision": args.precision,
           "config": {"workload": workload_desc(prob, args.traj, args.block),
                      "l2": "flushed between steps (256 MB write)",
                      "parallelism": "replicas" if world > 1 else "single GPU"},
           "terms_per_s": value * prob.terms_per_forward(),
           "leapfrog_steps_per_s": world * K * args.traj / (total_ms / 1000.0),
           "err_vs_fp64": err, "sampler": sampler, "precond_build_s": t_pc, "forms": forms,
           "roofline": roofline, "cpu_baseline": cpu, "e2e": e2e, "gpu_launches": int(launches), "clocks": clk,
           "cfg3": cfg3}
    h.close()
    return out


def main():
    args = parse()
    if args.impl == "reference":
        run_reference(args)
        return
    if args.config == "cfg2":
        main_batch(args)
        return
    args.precision = args.precision or "fp16x3"
    import torch
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    from paper_2504_07090_gb300 import build
    build.build()
    eps_arg = args.eps
    args.eps = eps_arg or EPS_DEFAULT.get(args.config, 0.01)
    head = measure(args, args.config, args.steps, args.warmup, rank, world, dist, local)
    big = None
    if args.config == "cfg1" and not args.no_cfg4:
        # the largest workload (127 antennas, 128 channels, 120 LSTs, 98,304 pixels), same
        # measurement with fewer timed steps; errors from visibilities sampled one by one
        a4 = argparse.Namespace(**vars(args))
        a4.eps = eps_arg or EPS_DEFAULT["cfg4"]
        big = measure(a4, "cfg4", max(1, min(args.steps, 3)), max(3, min(args.warmup, 3)), rank, world, dist, local,
                      forms_on=False, err_mode="sampled")
    comp = None
    if args.config == "cfg1" and not args.no_legendre:
        # cfg1 with the sky compressed onto 6 Legendre orders in frequency (Eq. fg_legendre):
        # 98,600 parameters, the same contraction kernels on the expanded channel modes
        ak = argparse.Namespace(**vars(args))
        ak.eps = eps_arg or EPS_DEFAULT["cfg1"]
        ak.no_cpu_baseline = True
        comp = measure(ak, "cfg1", max(1, min(args.steps, 5)), max(3, min(args.warmup, 3)), rank, world, dist, local,
                       forms_on=False, err_mode="sampled", freq_modes=LEGENDRE_ORDERS)
    batch = None
    if args.config == "cfg1" and not args.no_cfg2 and rank == 0:
        a2 = argparse.Namespace(**vars(args))
        a2.precision, a2.eps = None, None
        batch = measure_batch(a2, max(1, min(args.steps, 3)), 3)
        for k in ("metric", "n_gpus", "higher_is_better", "scaling", "vs_baseline", "data", "dtype"):
            batch.pop(k, None)
    if rank == 0:
        line = {"metric": METRIC, "value": head["value"], "unit": "chi2+grad evals/s", "n_gpus": world,
                "steps": args.steps, "warmup": args.warmup, "ms_per_step": head["ms_per_step"],
                "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
                "precision": args.precision, "data": "synthetic"}
        for k in ("config", "terms_per_s", "leapfrog_steps_per_s", "err_vs_fp64", "sampler", "precond_build_s",
                  "forms", "roofline", "cpu_baseline", "e2e", "gpu_launches", "clocks"):
            line[k] = head[k]
        if head.get("cfg3") is not None:
            line["cfg3"] = head["cfg3"]
        if big is not None:
            big.pop("forms", None)
            big.pop("cfg3", None)
            line["cfg4"] = big
        if comp is not None:
            comp.pop("forms", None)
            comp.pop("cfg3", None)
            comp.pop("cpu_baseline", None)
            line["cfg1_legendre"] = comp
        if batch is not None:
            line["cfg2"] = batch
        print(json.dumps(line), flush=True)
    if dist:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
