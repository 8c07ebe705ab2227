"""Benchmark of the CRL update step (arXiv 2408.11052, Algorithm 1 update body).

One step = insert one time slice for all environments -> sample + relabel a
batch -> critic step (encoders, energy + InfoNCE + penalty, backward, Adam)
-> actor step (policy, objective, backward, Adam), through the library's
public call crl_update_step.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
                  [--workload large|humanoid|ant|small|sweep] [--precision bf16|fp32|fp64]
                  [--path fused|plain] [--trace auto|gemm|energy|relabel|adam|aux|insert]
                  [--no-comparator] [--no-relabel] [--no-cpu-baseline] [--no-extra] [--no-error]

The headline is the BF16 fused path on the large-batch workload (batch 8192,
repr 256, 2 x 512 encoders); the FP32 plain path runs on the same workload in
the same process as "comparator".  "error" states the loss and per-tensor
gradient error of both arms against the FP64 oracle on one batch of the timed
workload.  "workloads" repeats the measurement on the Humanoid (batch 1024,
4 x 1024 LayerNorm encoders, critic + actor) and Ant (batch 256) workloads and
on the 32-agent sweep.  "relabel" reports the standalone sample + relabel
kernel at 2^20 and 2^22 samples per launch on Humanoid-shaped rows (its HBM
roofline).

Prints one JSON line (rank 0).  Under torchrun (N > 1) every rank runs its own
independent agent (its own Philox key and buffer): weak scaling, no data-path
collective; timing takes the max over ranks.
"""

import argparse
import json
import os
import statistics
import subprocess
import sys
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

from paper_2408_11052_gb300 import workload  # noqa: E402

WORKLOADS = {"ant": workload.ANT_AUTOGRAD, "small": workload.SMALL_FP32, "humanoid": workload.HUMANOID_BF16,
             "large": workload.LARGE_BATCH}
METRIC = "CRL update steps/sec and relabeled samples/sec, BF16 fused vs FP32 plain at stated error"
L2_FLUSH_BYTES = 256 << 20         # > 129 MB L2
FP32_ALU_PEAK_TFLOPS = 152 * 128 * 2 * 2.070e9 / 1e12   # SMs x FP32 lanes x 2 flop x max SM clock


def load_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f), "measured"
    except OSError:
        return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "bf16_tflops_sustained": 1700.0}, "fallback"


class ClockSampler:
    """nvidia-smi clock / throttle samples while the timed region runs."""
    QUERY = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device_index):
        self.idx = device_index
        self.proc = None

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.idx), f"--query-gpu={self.QUERY}",
                                          "--format=csv,noheader,nounits", "-lms", "100"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except OSError:
            self.proc = None
        time.sleep(0.3)
        return self

    def __exit__(self, *exc):
        self.lines = []
        if self.proc is not None:
            time.sleep(0.2)
            self.proc.terminate()
            try:
                out, _ = self.proc.communicate(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()
                out, _ = self.proc.communicate()
            self.lines = [l for l in out.splitlines() if l.strip()]
        return False

    def summary(self):
        sm, mx, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in getattr(self, "lines", []):
            f = [x.strip() for x in line.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                mx = float(f[2])
            except ValueError:
                continue
            for name, v in zip(names, f[5:9]):
                if v.lower() == "active":
                    reasons.add(name)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": mx, "reasons": sorted(reasons),
                "samples": len(sm)}


def dist_setup(n_gpus):
    import torch
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    else:
        torch.cuda.set_device(0)
    return rank, world, local


def barrier(world):
    if world > 1:
        import torch.distributed as dist
        dist.barrier()


def max_over_ranks(x, world):
    """The maximum of x over all ranks (NCCL on the GPU, gloo on the host)."""
    if world == 1:
        return x
    import torch
    import torch.distributed as dist
    device = "cuda" if dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([x], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def cpu_oracle_rate(w, n_steps, budget_s=20.0):
    """The FP64 oracle's update step on this host's cores: (steps/s, steps done, cores)."""
    import oracle
    nets = workload.init_agent(w)
    nets = {k: [{kk: vv.astype(np.float64) for kk, vv in l.items()} for l in v] for k, v in nets.items()}
    buf = oracle.relabel.ReplayBuffer(w.E, w.T, w.D, w.A)
    obs, act, done = buffer_contents_cached(w)
    buf.insert(obs, act, done)
    n_steps = min(n_steps, 64)
    extra = buffer_contents_cached(w, n=n_steps, seed_offset=1)
    state = oracle.step.AgentState(nets["phi"], nets["psi"], nets["pi"])
    cfg = dict(seed=w.seed, agent=0, B=w.B, goal_idx=w.goals(), gamma=w.gamma, energy=w.energy, tau=w.tau,
               loss=w.loss, sym_reduction=w.sym_reduction, beta=w.beta, penalty_axis=w.penalty_axis, alpha=w.alpha,
               lr_critic=w.lr_critic, lr_actor=w.lr_actor, alpha_autotune=w.alpha_autotune,
               target_entropy=-w.A if w.target_entropy is None else w.target_entropy,
               lr_alpha=w.lr_actor if w.lr_alpha is None else w.lr_alpha)
    done_steps = 0
    t0 = time.perf_counter()
    for i in range(n_steps):
        buf.insert(extra[0][i:i + 1], extra[1][i:i + 1], extra[2][i:i + 1])
        eps = oracle.actor.gaussian_noise(w.seed, 0, i, w.B, w.A)
        oracle.step.update_step(state, buf, cfg, i, eps)
        done_steps += 1
        if time.perf_counter() - t0 > budget_s:
            break
    dt = time.perf_counter() - t0
    cores = os.cpu_count()
    try:
        from threadpoolctl import threadpool_info
        info = threadpool_info()
        if info:
            cores = max(i.get("num_threads", 1) for i in info)
    except ImportError:
        pass
    return done_steps / dt, done_steps, cores


# The benchmark spec's error bars (FP32 path: relative errors; BF16 path: loss
# relative error and per-tensor gradient cosine), each against the FP64 oracle.
ERROR_BARS = {"fp32": {"loss_rel": 1e-5, "grad_rel": 1e-4}, "bf16": {"loss_rel": 2e-2, "grad_cos": 0.999}}


def oracle_error(w, dev, arms, step=0):
    """Oracle leg: the error of each arm's critic and actor step against the FP64
    oracle on one batch of the timed workload (its networks and buffer, relabel
    step `step`, actor noise given).  Per arm: the relabel indices (bit-exact or
    not), the loss parts' relative errors, and per parameter tensor the
    gradient's relative L2 error and cosine.  Runs outside every timed region."""
    import torch
    import oracle
    from paper_2408_11052_gb300 import api

    f32 = lambda x: float(np.float32(x))  # noqa: E731  (hyperparameters as the library holds them)
    tau, beta, alpha = f32(w.tau), f32(w.beta), f32(w.alpha)
    nets = workload.init_agent(w)
    n64 = {k: [{kk: vv.astype(np.float64) for kk, vv in l.items()} for l in v] for k, v in nets.items()}
    obs, act, done = buffer_contents_cached(w)
    buf = oracle.relabel.ReplayBuffer(w.E, w.T, w.D, w.A)
    buf.insert(obs, act, done)
    t0 = time.perf_counter()
    s, a, g, idx = oracle.relabel.sample_relabel(buf, w.seed, 0, step, w.B, w.goals(), w.gamma)
    parts, gphi, gpsi, _, _ = oracle.step.critic_loss_and_grad(n64["phi"], n64["psi"], s, a, g, w.energy, tau,
                                                               w.loss, w.sym_reduction, beta, w.penalty_axis)
    eps = workload.actor_noise(w.B, w.A, 3)
    ref_a = oracle.actor.actor_loss_and_grad(n64["pi"], n64["phi"], n64["psi"], s, g, eps.astype(np.float64),
                                             w.energy, tau, alpha)
    oracle_s = time.perf_counter() - t0

    def kink_units(net, x, rel=1e-6):
        """Hidden units whose pre-activation lies within rel x its layer's RMS of the
        ReLU kink in the oracle's forward: FP32 arithmetic may put them on either side."""
        _, cache = oracle.mlp.forward(net, x)
        return int(sum((np.abs(c["u"]) < rel * np.sqrt((c["u"] ** 2).mean())).sum() for c in cache[:-1]))

    kinks = {"phi": kink_units(n64["phi"], np.concatenate([s, a], 1)), "psi": kink_units(n64["psi"], g),
             "pi": kink_units(n64["pi"], np.concatenate([s, g], 1)),
             "phi_at_policy_action": kink_units(n64["phi"], np.concatenate([s, ref_a["a_new"]], 1)),
             "threshold": "|pre-activation| < 1e-6 x its layer's RMS in the FP64 forward (FP32 may flip the ReLU)"}

    def tensors(got, ref, net):
        rows = []
        for li, (gl, rl) in enumerate(zip(got, ref)):
            for k in rl:
                x, y = np.asarray(gl[k], np.float64).ravel(), np.asarray(rl[k], np.float64).ravel()
                nx, ny = np.linalg.norm(x), np.linalg.norm(y)
                rows.append({"tensor": f"{net}.{li}.{k}", "rel_err": float(np.linalg.norm(x - y) / (ny or 1.0)),
                             "cos": float(x @ y / (nx * ny)) if nx > 0 and ny > 0 else float(nx == ny)})
        return rows

    out = {"workload": w.name, "batch": f"relabel step {step} of the timed workload's buffer and networks",
           "oracle": "FP64 numpy, materialised B x B", "oracle_s": oracle_s, "bars": ERROR_BARS,
           "kink_units": kinks}
    for precision, path in arms:
        ctx = api.CRLContext(w, precision=precision, path=path)
        for k, v in nets.items():
            ctx.load_network(k, v)
        ctx.insert(torch.from_numpy(obs).to(dev), torch.from_numpy(act).to(dev), torch.from_numpy(done).to(dev))
        sd, ad, gd, idd = ctx.sample(step=step)
        lc = ctx.critic_step(sd, ad, gd, apply_update=False).cpu().numpy()
        la = ctx.actor_step(sd, gd, torch.from_numpy(eps).to(dev), apply_update=False).cpu().numpy()
        torch.cuda.synchronize()
        rc, status = ctx.sync_status()
        rel = lambda x, y: abs(float(x) - float(y)) / (abs(float(y)) or 1.0)  # noqa: E731
        grads = tensors(ctx.network("phi", "grads"), gphi, "phi") + tensors(ctx.network("psi", "grads"), gpsi, "psi") \
            + tensors(ctx.network("pi", "grads"), ref_a["grads"], "pi")
        key = "bf16" if precision == "bf16" else "fp32"
        r = {"precision": precision, "path": path, "status": status,
             "relabel_indices_exact": bool(np.array_equal(idd.cpu().numpy().astype(np.int64), idx)),
             "loss_rel_err": {"critic_total": rel(lc[0], parts["total"]), "critic_fwd": rel(lc[1], parts["fwd"]),
                              "critic_bwd": rel(lc[2], parts["bwd"]), "penalty": rel(lc[3], parts["penalty"]),
                              "actor": rel(la[0], ref_a["loss"])},
             "grad_worst_rel_err": max(t["rel_err"] for t in grads),
             "grad_worst_cos": min(t["cos"] for t in grads), "grads": grads}
        bar = ERROR_BARS[key]

        def within(tensors, losses):
            loss_ok = max(r["loss_rel_err"][k] for k in losses) <= bar["loss_rel"]
            if key == "bf16":
                return loss_ok and min(t["cos"] for t in tensors) >= bar["grad_cos"]
            return loss_ok and max(t["rel_err"] for t in tensors) <= bar["grad_rel"]

        crit_t = [t for t in grads if not t["tensor"].startswith("pi.")]
        actor_t = [t for t in grads if t["tensor"].startswith("pi.")]
        r["within_bars_critic"] = bool(within(crit_t, ("critic_total", "critic_fwd", "critic_bwd", "penalty")))
        r["within_bars_actor"] = bool(within(actor_t, ("actor",)))
        r["within_bars"] = bool(r["within_bars_critic"] and r["within_bars_actor"] and r["relabel_indices_exact"]
                                and rc == api.OK)
        out[f"{precision}_{path}"] = r
        ctx.close()
    return out


BLAS_THREAD_VARS = ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS", "BLIS_NUM_THREADS")


def cpu_oracle_rate_one_thread(args, budget_s=10.0):
    """The same oracle rate in a child process whose BLAS runs one thread:
    (steps/s, steps done), or None when the child fails."""
    cmd = [sys.executable, os.path.abspath(__file__), "--oracle-rate", str(budget_s), "--workload", args.workload]
    for flag, v in (("--loss", args.loss), ("--energy", args.energy)):
        if v is not None:
            cmd += [flag, v]
    if args.alpha_autotune:
        cmd.append("--alpha-autotune")
    env = dict(os.environ, **{k: "1" for k in BLAS_THREAD_VARS})
    try:
        out = subprocess.run(cmd, env=env, capture_output=True, text=True, timeout=budget_s + 300)
        r = json.loads(out.stdout.strip().splitlines()[-1])
        return r["value"], r["steps"]
    except (subprocess.SubprocessError, ValueError, KeyError, IndexError):
        return None


def run_reference(args, w):
    """--impl reference: the FP64 CPU oracle, as it stands, on the host cores."""
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    n = args.warmup + args.steps
    rate, steps, cores = cpu_oracle_rate(w, n, budget_s=240.0)
    line = {"impl": "reference", "metric": METRIC, "value": rate, "unit": "update steps/s", "n_gpus": 0,
            "steps": steps, "warmup": 0, "ms_per_step": 1e3 / rate, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic (seeded random-walk buffer, random-init nets)",
            "samples_per_s": rate * w.B,
            "config": {"workload": w.name, "batch": w.B, "envs": w.E, "steps_per_env": w.T,
                       "sample": f"{steps} full update steps (insert+relabel+critic+actor+Adam) of the workload"},
            "cpu_baseline": {"value": rate, "unit": "update steps/s", "cores": cores, "kind": "oracle",
                             "sample": f"{steps} update steps"},
            "e2e": {"value": rate, "unit": "update steps/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


RELABEL_ROWS = workload.Workload("relabel_humanoid_rows_E1024xT1000_D268_A17_G3", E=1024, T=1000, D=268, A=17,
                                 G=3, B=256, hidden=64, layers=1, repr=64, seed=5)


def traffic_record(kernel_class, workload_name, precision, path):
    """DRAM bytes per launch of the dominant kernel class from the committed ncu
    summary, or None when the summary is missing or its kernel source changed."""
    import hashlib
    try:
        with open(os.path.join(ROOT, "profiles", "roofline_traffic.json")) as f:
            table = json.load(f)
    except OSError:
        return None
    rec = table.get(f"{kernel_class}|{workload_name}|{precision}|{path}")
    if rec is None:
        return None
    h = hashlib.sha256()
    for rel in rec["sources"]:
        with open(os.path.join(ROOT, rel), "rb") as f:
            h.update(f.read())
    return rec["bytes_per_launch"] if h.hexdigest() == rec["sources_sha256"] else None


_BUFFERS = {}


def buffer_contents_cached(w, n=None, seed_offset=0):
    """workload.buffer_contents (fixed-length episodes), generated once per
    (workload, n, seed offset) and reused by every arm of this run."""
    key = (w.name, w.E, w.T, w.D, w.A, n, seed_offset)
    if key not in _BUFFERS:
        _BUFFERS[key] = workload.buffer_contents(w, n=n, mean_len=None, seed_offset=seed_offset)
    return _BUFFERS[key]


def roofline_of(arm, w, precision, path):
    """The roofline object of an arm's traced kernel class: algorithmic work per
    launch over the launches' CUDA-event time, against the measured peak."""
    peaks, peak_src = load_peaks()
    cls = arm["trace_class"]
    n_tr, tr_ms, tr_work = arm["trace"]
    traffic = traffic_record(cls, w.name, precision, path)
    common = {"kernel_class": cls, "launches": n_tr, "avg_launch_us": 1e3 * tr_ms / max(n_tr, 1),
              "work_per_launch": tr_work / max(n_tr, 1),
              "timing": "eager traced pass of the same K steps (CUDA events around every launch of the class)",
              "traffic": traffic}
    if cls in ("gemm", "energy") and precision == "bf16":
        achieved = tr_work / (tr_ms / 1e3) / 1e12
        peak = peaks["bf16_tflops_sustained"]
        roof = {"bound": "tensor", "achieved": achieved, "peak": peak, "unit": "TFLOP/s", "frac": achieved / peak,
                "peak_source": f"{peak_src} bf16_tflops_sustained (kernel timed inside a long step)", **common}
        per_launch = tr_work / max(n_tr, 1)
        # at the peak a launch's work takes per_launch / peak; when that is far
        # below the launch's duration, the launch is latency-bound, not tensor-bound
        roof["note"] = (f"{per_launch / 1e6:.1f} MFLOP per launch = {per_launch / (peak * 1e12) * 1e6:.2f} us at the "
                        f"peak against {1e3 * tr_ms / max(n_tr, 1):.1f} us measured")
        tuned = arm.get("gemm_tuning")
        if cls == "gemm" and tuned:
            # the tensor work as launched (the forward layers multiply BF16 hi / lo
            # pairs), each tuned group once per step, over the same traced time
            alg = sum(g["gflop"] for g in tuned)
            issued = sum(g.get("issued_gflop", g["gflop"]) for g in tuned)
            if alg > 0:
                rate = achieved * issued / alg
                roof["issued"] = {"tflops": rate, "frac": rate / peak, "per_algorithmic": issued / alg,
                                  "note": "tensor work as launched: the forward layers' BF16 hi / lo input and "
                                          "weight products (two to four per algorithmic product), from the "
                                          "autotuner report, over the same traced launches"}
    elif cls in ("gemm", "energy"):
        achieved = tr_work / (tr_ms / 1e3) / 1e12
        roof = {"bound": "alu", "achieved": achieved, "peak": FP32_ALU_PEAK_TFLOPS, "unit": "TFLOP/s",
                "frac": achieved / FP32_ALU_PEAK_TFLOPS,
                "peak_source": "derived: 152 SMs x 128 FP32 lanes x 2 flop x 2070 MHz", **common}
    else:
        achieved = tr_work / (tr_ms / 1e3) / 1e9
        roof = {"bound": "hbm", "achieved": achieved, "peak": peaks["hbm_gbs"], "unit": "GB/s",
                "frac": achieved / peaks["hbm_gbs"], "peak_source": f"{peak_src} hbm_gbs", **common}
    if traffic is not None:
        roof["traffic_source"] = "profiles/roofline_traffic.json (ncu dram__bytes_read.sum + dram__bytes_write.sum)"
    return roof


def secondary(args, w, dev, flush, steps, error):
    """One more workload on one GPU: the BF16 fused arm (breakdown, dominant
    class roofline, host-input e2e) next to the FP32 plain arm, and (error) the
    oracle leg's error table for both."""
    sub = argparse.Namespace(**vars(args))
    sub.steps, sub.trace = steps, "auto"
    a = run_arm(sub, w, "bf16", "fused", dev, 1, 0, flush, full=True)
    c = run_arm(sub, w, "fp32", "plain", dev, 1, 0, flush, full=False)
    v, cv = steps / (a["ms"] / 1e3), steps / (c["ms"] / 1e3)
    out = {"workload": w.name, "value": v, "unit": "update steps/s", "ms_per_step": a["ms"] / steps, "steps": steps,
           "samples_per_s": v * w.B, "precision": "bf16", "path": "fused",
           "e2e": {"value": steps / (a["e2e_ms"] / 1e3), "unit": "update steps/s",
                   "h2d_bytes_per_step": w.E * (w.D + w.A) * 4 + w.E, "d2h_bytes_per_step": 24},
           "comparator": {"precision": "fp32", "path": "plain", "value": cv, "unit": "update steps/s",
                          "ms_per_step": c["ms"] / steps, "speedup": v / cv},
           "launches_per_step": a["launches_per_step"],
           "breakdown": {"timing": "eager, events around every launch", **a["breakdown"]},
           "roofline": roofline_of(a, w, "bf16", "fused"), "clocks": a["clocks"]}
    if error:
        out["error"] = oracle_error(w, dev, (("bf16", "fused"), ("fp32", "plain")))
    return out


def run_arm(args, w, precision, path, dev, world, rank, flush, full):
    """Prefill, warm up and time one configuration of the update step.  full:
    also the traced roofline pass, the end-to-end (host-buffer) pass and the
    launch count."""
    import torch
    from paper_2408_11052_gb300 import api

    stream = torch.cuda.current_stream()
    ctx = api.CRLContext(w, precision=precision, path=path, agent=rank)
    for k, v in workload.init_agent(w).items():
        ctx.load_network(k, v)
    obs, act, done = buffer_contents_cached(w, seed_offset=rank)
    ctx.insert(torch.from_numpy(obs).to(dev), torch.from_numpy(act).to(dev), torch.from_numpy(done).to(dev))
    del obs, act, done
    n_all = args.warmup + 2 * args.steps + 8
    ins = buffer_contents_cached(w, n=n_all, seed_offset=100 + rank)
    d_obs, d_act, d_done = (torch.from_numpy(x).to(dev) for x in ins)
    h_obs, h_act, h_done = (torch.from_numpy(x).pin_memory() for x in ins)
    loss_dev = torch.zeros(6, dtype=torch.float32, device=dev)
    loss_host = torch.zeros(6, dtype=torch.float32).pin_memory()
    cursor = [0]

    def step_device():
        i = cursor[0]
        cursor[0] += 1
        ctx.update_step(d_obs[i:i + 1], d_act[i:i + 1], d_done[i:i + 1], loss_out=loss_dev)

    def step_host():
        i = cursor[0]
        cursor[0] += 1
        ctx.update_step(h_obs[i:i + 1].numpy(), h_act[i:i + 1].numpy(), h_done[i:i + 1].numpy(), loss_out=loss_host)

    def timed(fn, K, trace=None):
        starts = [torch.cuda.Event(enable_timing=True) for _ in range(K)]
        ends = [torch.cuda.Event(enable_timing=True) for _ in range(K)]
        barrier(world)
        torch.cuda.synchronize()
        if trace:
            ctx.trace_start(trace, 64 * K)
        for k in range(K):
            flush.fill_(k & 0xFF)                 # evict L2 between steps (not timed)
            starts[k].record(stream)
            fn()
            ends[k].record(stream)
        torch.cuda.synchronize()
        barrier(world)
        tr = ctx.trace_stop() if trace else None
        ms = sum(s.elapsed_time(e) for s, e in zip(starts, ends))
        return ms, tr

    def timed_e2e(K):
        """Host wall clock around each step with host inputs and a host read of
        its loss (the step's result): the host waits for every step."""
        total = 0.0
        for k in range(K):
            flush.fill_(k & 0xFF)                 # evict L2 between steps (not timed)
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            step_host()
            stream.synchronize()
            _ = float(loss_host[0])
            total += time.perf_counter() - t0
        return 1e3 * total

    for _ in range(args.warmup):
        step_device()
    torch.cuda.synchronize()
    rc, status = ctx.sync_status()
    assert rc == api.OK, f"warm-up status {status}"
    out = {}
    if full:
        # kernels per step and the time of each kernel class: every class traced
        # over 20 eager steps (CUDA events around each of its launches)
        launches, breakdown = 0, {}
        for cls in api.TRACE:
            ctx.trace_start(cls, 4096)
            for _ in range(20):
                step_device()
            n, cls_ms, _ = ctx.trace_stop()
            launches += n // 20
            breakdown[cls] = {"launches_per_step": n // 20, "us_per_step": 1e3 * cls_ms / 20,
                              "us_per_launch": 1e3 * cls_ms / max(n, 1)}
        out["launches_per_step"] = launches
        out["breakdown"] = breakdown
        # the roofline's kernel class: the one that takes the most time per step
        out["trace_class"] = args.trace if args.trace != "auto" else \
            max(breakdown, key=lambda c: breakdown[c]["us_per_step"])

    # timed region: graph-replayed steps, no tracing (tracing forces eager launches)
    with ClockSampler(dev.index) as clk:
        ms, _ = timed(step_device, args.steps)
    out["ms"] = max_over_ranks(ms, world)
    out["clocks"] = clk.summary()
    if full:
        # roofline pass: the same K steps again, eager, with CUDA events around
        # every launch of the traced kernel class
        _, out["trace"] = timed(step_device, args.steps, trace=out["trace_class"])
        for _ in range(3):
            step_host()
        barrier(world)
        e2e_ms = timed_e2e(args.steps)
        barrier(world)
        out["e2e_ms"] = max_over_ranks(e2e_ms, world)
    rc, status = ctx.sync_status()
    assert rc == api.OK, f"status {status}"
    if full and precision == "bf16":
        out["gemm_tuning"] = api.gemm_tuning_report(ctx.handle)
    ctx.close()
    return out


def collect_loop(w, precision, path, dev, unroll=62, utd=16, rounds=1):
    """Algorithm 1's outer loop with the collection stub: each round collects
    `unroll` synthetic environment steps for all E environments (crl_collect),
    then runs E * unroll / utd update steps (App. B.3: 1024 environments, unroll
    62; §4.1 and §5.6: update-to-data ratio 1:16).  One warm-up round, then
    `rounds` timed rounds (CUDA events on the stream)."""
    import torch
    from paper_2408_11052_gb300 import api

    stream = torch.cuda.current_stream()
    ctx = api.CRLContext(w, precision=precision, path=path)
    for k, v in workload.init_agent(w).items():
        ctx.load_network(k, v)
    updates = w.E * unroll // utd
    loss = torch.zeros(6, dtype=torch.float32, device=dev)
    ctx.collect(max(unroll, 64), w.T)            # prefill before the first update
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(3 * (rounds + 1))]
    for r in range(rounds + 1):
        ev[3 * r].record(stream)
        ctx.collect(unroll, w.T)
        ev[3 * r + 1].record(stream)
        for _ in range(updates):
            ctx.update_step(loss_out=loss)
        ev[3 * r + 2].record(stream)
    torch.cuda.synchronize()
    rc, status = ctx.sync_status()
    assert rc == api.OK, f"collect loop status {status}"
    col = sum(ev[3 * r].elapsed_time(ev[3 * r + 1]) for r in range(1, rounds + 1)) / rounds
    upd = sum(ev[3 * r + 1].elapsed_time(ev[3 * r + 2]) for r in range(1, rounds + 1)) / rounds
    env_steps = w.E * unroll
    return {"env_steps_per_s": env_steps / ((col + upd) / 1e3), "update_steps_per_s": updates / ((col + upd) / 1e3),
            "envs": w.E, "unroll": unroll, "utd": f"1:{utd}", "updates_per_round": updates,
            "collect_ms_per_round": col, "update_ms_per_round": upd, "rounds_timed": rounds,
            "episode_length": w.T, "precision": precision, "path": path,
            "note": "collection = crl_collect (synthetic dynamics standing in for the simulator, policy forward "
                    "on all envs, insert); updates = crl_update_step graph replays"}


def relabel_throughput(dev, flush, sizes=(1 << 20, 1 << 22), K=10, W=3):
    """Standalone sample + relabel launches on Humanoid-shaped rows (HBM-bound):
    samples/s and achieved GB/s per batch size."""
    import torch
    from paper_2408_11052_gb300 import api

    w = RELABEL_ROWS
    stream = torch.cuda.current_stream()
    ctx = api.CRLContext(w, precision="fp32")
    obs, act, done = workload.buffer_contents(w, mean_len=None)
    ctx.insert(torch.from_numpy(obs).to(dev), torch.from_numpy(act).to(dev), torch.from_numpy(done).to(dev))
    del obs, act, done
    per = (w.D + w.A + 1 + w.G) * 4 + (w.D + w.A + w.G) * 4   # read row + episode end + goal dims, write s, a, g
    res = []
    for n in sizes:
        kw = dict(dtype=torch.float32, device=dev)
        out = (torch.empty(n, w.D, **kw), torch.empty(n, w.A, **kw), torch.empty(n, w.G, **kw), None)
        for i in range(W):
            ctx.sample(step=i, B=n, out=out)
        starts = [torch.cuda.Event(enable_timing=True) for _ in range(K)]
        ends = [torch.cuda.Event(enable_timing=True) for _ in range(K)]
        torch.cuda.synchronize()
        for k in range(K):
            flush.fill_(k & 0xFF)
            starts[k].record(stream)
            ctx.sample(step=100 + k, B=n, out=out)
            ends[k].record(stream)
        torch.cuda.synchronize()
        ms = sum(s.elapsed_time(e) for s, e in zip(starts, ends)) / K
        res.append({"samples_per_launch": n, "value": n / (ms / 1e3), "unit": "samples/s", "us_per_launch": 1e3 * ms,
                    "achieved_gbs": per * n / (ms / 1e3) / 1e9,
                    "bytes_per_sample": per})
        del out
    rc, status = ctx.sync_status()
    assert rc == api.OK, f"relabel status {status}"
    ctx.close()
    return w, res


def run_sweep_arm(args, ws, precision, path, grouped, dev, flush, steps, full):
    """A batched sweep of independent agents: sweep steps/s (and, with full,
    the traced roofline pass, host-input pass and launch count)."""
    import torch
    from paper_2408_11052_gb300 import api

    stream = torch.cuda.current_stream()
    sw = api.CRLSweep(ws, precision, path, grouped=grouped)
    n_all = 64                      # insert slices cycled through (the values do not change the work)
    ins = []
    for i, w in enumerate(ws):
        for k, v in workload.init_agent(w).items():
            sw.agents[i].load_network(k, v)
        obs, act, done = workload.buffer_contents_device(w, device=dev)
        sw.agents[i].insert(obs, act, done)
        del obs, act, done
        ins.append(workload.buffer_contents_device(w, n=n_all, seed_offset=100, device=dev))
    host = None
    if full:
        host = [tuple(x.cpu().pin_memory() for x in a) for a in ins]
    loss_dev = torch.zeros(len(ws), 6, dtype=torch.float32, device=dev)
    loss_host = torch.zeros(len(ws), 6, dtype=torch.float32).pin_memory()
    cursor = [0]

    def step(src, loss):
        i = cursor[0] % n_all
        cursor[0] += 1
        sw.update_step([a[0][i:i + 1] for a in src], [a[1][i:i + 1] for a in src], [a[2][i:i + 1] for a in src],
                       loss_out=loss)

    def timed(fn, K, trace=None):
        starts = [torch.cuda.Event(enable_timing=True) for _ in range(K)]
        ends = [torch.cuda.Event(enable_timing=True) for _ in range(K)]
        torch.cuda.synchronize()
        if trace:
            sw.agents[0].trace_start(trace, 4096 * K)
        for k in range(K):
            flush.fill_(k & 0xFF)
            starts[k].record(stream)
            fn()
            ends[k].record(stream)
        torch.cuda.synchronize()
        tr = sw.agents[0].trace_stop() if trace else None
        return sum(s.elapsed_time(e) for s, e in zip(starts, ends)), tr

    for _ in range(args.warmup):
        step(ins, loss_dev)
    torch.cuda.synchronize()
    rc, status = sw.sync_status()
    assert rc == api.OK, f"sweep warm-up status {status}"
    out = {}
    with ClockSampler(dev.index) as clk:
        out["ms"], _ = timed(lambda: step(ins, loss_dev), steps)
    out["clocks"] = clk.summary()
    if full:
        launches = 0
        for cls in api.TRACE:
            sw.agents[0].trace_start(cls, 1 << 16)
            step(ins, loss_dev)
            launches += sw.agents[0].trace_stop()[0]
        out["launches_per_step"] = launches
        _, out["trace"] = timed(lambda: step(ins, loss_dev), min(steps, 20), trace=args.trace)
        for _ in range(3):
            step(host, loss_host)
        out["e2e_ms"], _ = timed(lambda: step(host, loss_host), steps)
    rc, status = sw.sync_status()
    assert rc == api.OK, f"sweep status {status}"
    sw.close()
    return out


def run_sweep(args, dev, flush):
    """The batched-sweep workload: 32 independent agents (batch 256..2048, obs
    29 / 64 / 268, repr 64 / 128, 512 envs x 1000 steps each) per update step;
    the grouped BF16 sweep, with the same agents stepped one after another in
    BF16 and in FP32 as comparators."""
    ws = workload.sweep_agents(32)
    B_total = sum(w.B for w in ws)
    main_arm = run_sweep_arm(args, ws, "bf16", "fused", True, dev, flush, args.steps, full=True)
    comps = []
    if not args.no_comparator:
        from paper_2408_11052_gb300 import api
        prev = api.set_autotune(False)
        k = min(args.steps, 50)
        c = run_sweep_arm(args, ws, "bf16", "fused", True, dev, flush, k, full=False)
        api.set_autotune(prev)
        comps.append({"precision": "bf16", "path": "fused", "grouped": True, "autotune": False,
                      "value": len(ws) * k / (c["ms"] / 1e3), "unit": "agent update steps/s",
                      "ms_per_step": c["ms"] / k, "clocks": c["clocks"],
                      "note": "grouped, tile widths from the fixed rule instead of the autotuner"})
        for prec, path in (("bf16", "fused"), ("fp32", "plain")):
            k = min(args.steps, 20)
            c = run_sweep_arm(args, ws, prec, path, False, dev, flush, k, full=False)
            comps.append({"precision": prec, "path": path, "grouped": False,
                          "value": len(ws) * k / (c["ms"] / 1e3), "unit": "agent update steps/s",
                          "ms_per_step": c["ms"] / k, "clocks": c["clocks"],
                          "note": "the same agents' update steps one after another in one CUDA graph"})
    ms = main_arm["ms"]
    sweeps_per_s = args.steps / (ms / 1e3)
    value = len(ws) * sweeps_per_s
    for c in comps:
        c["speedup"] = value / c["value"]
    peaks, peak_src = load_peaks()
    n_tr, tr_ms, tr_work = main_arm["trace"]
    achieved = tr_work / (tr_ms / 1e3) / 1e12
    peak = peaks["bf16_tflops_sustained"]
    roof = {"bound": "tensor", "achieved": achieved, "peak": peak, "unit": "TFLOP/s", "frac": achieved / peak,
            "kernel_class": args.trace, "launches": n_tr, "avg_launch_us": 1e3 * tr_ms / max(n_tr, 1),
            "timing": "eager traced pass (CUDA events around every launch of the class)", "traffic": None,
            "peak_source": f"{peak_src} bf16_tflops_sustained (kernel timed inside a long step)"}
    h2d = sum(w.E * (w.D + w.A) * 4 + w.E for w in ws)
    line = {"metric": METRIC, "value": value, "unit": "agent update steps/s", "n_gpus": 1, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms / args.steps, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "bf16", "data": "synthetic (seeded random-walk buffers, random-init nets)",
            "samples_per_s": B_total * sweeps_per_s,
            "config": {"workload": "sweep_32_agents_E512xT1000_B256-2048_D29-64-268_R64-128_2x256",
                       "agents": len(ws), "batch_total": B_total, "batches": [w.B for w in ws],
                       "obs": [w.D for w in ws], "repr": [w.repr for w in ws], "hidden": [256, 256],
                       "precision": "bf16", "path": "fused", "grouped": True,
                       "l2": "flushed between timed steps (256 MiB write, outside the events)",
                       "step": "per agent: insert 1 slice + relabel + critic + Adam + actor + Adam",
                       "parallelism": "32 independent agents on one GPU"},
            "e2e": {"value": len(ws) * args.steps / (main_arm["e2e_ms"] / 1e3), "unit": "agent update steps/s",
                    "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": 24 * len(ws)},
            "gpu_launches": main_arm["launches_per_step"] * args.steps,
            "roofline": roof, "clocks": main_arm["clocks"]}
    if comps:
        line["comparator"] = comps
    return line


def api_losses():
    from paper_2408_11052_gb300 import api as _api
    return _api.LOSS


def build_parser():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=200)
    ap.add_argument("--warmup", type=int, default=20)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="large", choices=sorted(WORKLOADS) + ["sweep"])
    ap.add_argument("--precision", default="bf16", choices=["fp32", "bf16", "fp64"])
    ap.add_argument("--path", default="fused", choices=["plain", "fused"])
    ap.add_argument("--trace", default="auto", choices=["auto", "gemm", "energy", "relabel", "adam", "aux", "insert"],
                    help="kernel class of the roofline object (auto: the one that takes the most time per step)")
    ap.add_argument("--no-extra", action="store_true",
                    help="skip the Humanoid, Ant and sweep measurements of the default large-batch run")
    ap.add_argument("--no-error", action="store_true", help="skip the error against the FP64 oracle")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-comparator", action="store_true", help="skip the FP32 plain arm")
    ap.add_argument("--no-relabel", action="store_true", help="skip the standalone relabel throughput")
    ap.add_argument("--no-loop", action="store_true", help="skip the collection + update loop (UTD 1:16)")
    ap.add_argument("--no-autotune", action="store_true",
                    help="fixed GEMM tile rule (deterministic launch sequence for profiler captures)")
    ap.add_argument("--only-relabel", action="store_true",
                    help="run only the standalone relabel throughput (a short command for ncu captures)")
    ap.add_argument("--loss", default=None, choices=sorted(api_losses()),
                    help="contrastive objective instead of the workload's (App. A.2 / §5.2)")
    ap.add_argument("--energy", default=None, choices=["l2", "dot", "cos", "l2sq", "l1"],
                    help="energy function instead of the workload's")
    ap.add_argument("--alpha-autotune", action="store_true", help="learn the entropy coefficient")
    ap.add_argument("--gemm-kernel", default="any", choices=["any", "one_tile", "persistent", "cta_pair"],
                    help="BF16 GEMM kernel family the autotuner may pick from")
    ap.add_argument("--oracle-rate", type=float, default=None, help=argparse.SUPPRESS)
    return ap


def main():
    args = build_parser().parse_args()
    args.warmup = max(args.warmup, 3)
    w = WORKLOADS.get(args.workload, workload.LARGE_BATCH)
    over = {k: v for k, v in (("loss", args.loss), ("energy", args.energy)) if v is not None}
    if args.alpha_autotune:
        over["alpha_autotune"] = True
    if over:
        w = w.with_(**over)
    if args.oracle_rate is not None:
        rate, steps, _ = cpu_oracle_rate(w, 200, budget_s=args.oracle_rate)
        print(json.dumps({"value": rate, "steps": steps}), flush=True)
        return
    if args.impl == "reference":
        run_reference(args, w)
        return

    import torch

    from paper_2408_11052_gb300 import api as _api
    if args.no_autotune:
        _api.set_autotune(False)
    _api.set_gemm_kernel(args.gemm_kernel)
    rank, world, local = dist_setup(args.gpus)
    dev = torch.device("cuda", local if world > 1 else 0)
    # one non-default stream for everything: the library replays the update step
    # as a CUDA graph there (the legacy default stream cannot be captured)
    torch.cuda.set_stream(torch.cuda.Stream(device=dev))
    flush = torch.empty(L2_FLUSH_BYTES, dtype=torch.uint8, device=dev)
    if args.workload == "sweep":
        print(json.dumps(run_sweep(args, dev, flush)), flush=True)
        return
    if args.only_relabel:
        rw, res = relabel_throughput(dev, flush)
        print(json.dumps({"relabel": {"workload": rw.name, "results": res}}), flush=True)
        return

    main_arm = run_arm(args, w, args.precision, args.path, dev, world, rank, flush, full=True)
    ms = main_arm["ms"]
    value = world * args.steps / (ms / 1e3)
    comparator = None
    if not args.no_comparator and (args.precision, args.path) != ("fp32", "plain"):
        comp = run_arm(args, w, "fp32", "plain", dev, world, rank, flush, full=False)
        cv = world * args.steps / (comp["ms"] / 1e3)
        comparator = {"precision": "fp32", "path": "plain", "value": cv, "unit": "update steps/s",
                      "ms_per_step": comp["ms"] / args.steps, "speedup": value / cv, "clocks": comp["clocks"],
                      "note": "same workload, timing and launch mode; plain SIMT FP32 kernels, B x B materialised"}

    roof = roofline_of(main_arm, w, args.precision, args.path)

    error = None
    if rank == 0 and world == 1 and not args.no_error:
        arms = [(args.precision, args.path)] + ([("fp32", "plain")] if comparator is not None else [])
        error = oracle_error(w, dev, arms)

    extra = None
    if rank == 0 and world == 1 and not args.no_extra and args.workload == "large" and not over:
        extra = {"humanoid": secondary(args, workload.HUMANOID_BF16, dev, flush, min(args.steps, 100),
                                       error=not args.no_error),
                 "ant": secondary(args, workload.ANT_AUTOGRAD, dev, flush, args.steps, error=not args.no_error)}
        sub = argparse.Namespace(**vars(args))
        sub.steps, sub.no_comparator, sub.trace = min(args.steps, 50), True, "gemm"
        extra["sweep"] = run_sweep(sub, dev, flush)

    loop_w = workload.ANT_AUTOGRAD if args.workload == "large" else w
    loop = None
    if rank == 0 and world == 1 and not args.no_loop:
        loop = collect_loop(loop_w, args.precision, args.path, dev)

    peaks, peak_src = load_peaks()
    relabel = None
    if rank == 0 and world == 1 and not args.no_relabel:
        rw, res = relabel_throughput(dev, flush)
        for r in res:
            r["roofline"] = {"bound": "hbm", "achieved": r["achieved_gbs"], "peak": peaks["hbm_gbs"], "unit": "GB/s",
                             "frac": r["achieved_gbs"] / peaks["hbm_gbs"], "peak_source": f"{peak_src} hbm_gbs"}
        relabel = {"workload": rw.name, "kernel": "relabel_kernel (crl_sample_relabel, one launch per batch)",
                   "l2": "flushed between launches", "results": res}

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        rate, steps, cores = cpu_oracle_rate(w, 200, budget_s=15.0)
        cpu = {"value": rate, "unit": "update steps/s", "cores": cores, "kind": "oracle",
               "sample": f"{steps} full update steps of the same workload (FP64 numpy oracle; its BLAS and its "
                         f"distance-energy row blocks on every host core)"}
        if rate > 0.5:        # one thread: only where a step takes well under a second on all cores
            one = cpu_oracle_rate_one_thread(args)
            if one is not None:
                cpu["one_thread"] = {"value": one[0], "unit": "update steps/s", "cores": 1,
                                     "sample": f"{one[1]} update steps, BLAS and row blocks on one thread"}
        else:
            cpu["one_thread"] = {"value": None, "note": f"skipped: one step takes {1 / rate:.0f} s on all cores"}

    h2d = w.E * (w.D + w.A) * 4 + w.E
    line = {"metric": METRIC, "value": value, "unit": "update steps/s", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms / args.steps, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": {"fp32": "f32", "bf16": "bf16", "fp64": "f64"}[args.precision],
            "data": "synthetic (seeded random-walk buffer, random-init nets)",
            "samples_per_s": value * w.B,
            "config": {"workload": w.name, "batch": w.B, "envs": w.E, "steps_per_env": w.T, "obs": w.D,
                       "action": w.A, "goal": w.G, "hidden": [w.hidden] * w.layers, "repr": w.repr,
                       "energy": w.energy, "loss": w.loss, "alpha_autotune": bool(w.alpha_autotune),
                       "precision": args.precision, "path": args.path,
                       "gemm_kernel": args.gemm_kernel,
                       "l2": "flushed between timed steps (256 MiB write, outside the events)",
                       "step": "insert 1 slice + relabel + critic fwd/bwd + Adam + actor fwd/bwd + Adam",
                       "parallelism": f"{world} independent agents"},
            "e2e": {"value": world * args.steps / (main_arm["e2e_ms"] / 1e3), "unit": "update steps/s",
                    "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": 24,
                    "timing": "host wall clock per step: pinned host inputs read by the insert kernel, the "
                              "loss copied to pinned host memory, the host waits for it every step"},
            "gpu_launches": main_arm["launches_per_step"] * args.steps,
            "breakdown": {"timing": "eager, events around every launch (no launch overlap): sums exceed ms_per_step",
                          **main_arm["breakdown"]},
            "roofline": roof,
            "clocks": main_arm["clocks"]}
    if main_arm.get("gemm_tuning") is not None:
        line["gemm_tuning"] = {"note": "the tile autotuner's picks for this workload's grouped GEMM launches, "
                                       "each candidate's faster time per launch over two timing rounds (us)",
                               "groups": main_arm["gemm_tuning"]}
    if comparator is not None:
        line["comparator"] = comparator
    if error is not None:
        line["error"] = error
    if extra is not None:
        line["workloads"] = extra
    if relabel is not None:
        line["relabel"] = relabel
    if loop is not None:
        line["collect_loop"] = loop
    if cpu is not None:
        line["cpu_baseline"] = cpu
    if rank == 0:
        print(json.dumps(line), flush=True)
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
