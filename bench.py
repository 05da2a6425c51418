"""Throughput of the batched joint lensing + dynamics log-likelihood on B300.

Default workload: the RXJ1131-scale system (200x200 image at 2x supersampling, EPL +
shear + SIS, two lens-light Sersics + Sersic source, 21x21 PSF; JAM with 20 mass +
2x10 light Gaussians + BH, 60x60 sky at 4x sub-sampling, GL32, 50 bins, 4 images),
a batch of 256 samples from the priors.  One step = one glad_loglike call over the
batch (every kernel of the path).  With --grad the step is glad_loglike_grad over
a batch of 64 samples.

Data: seeded synthetic inputs; the image and the binned v_rms are the library's own
model at the truth plus seeded noise, the quasar images sit on the Einstein ring.

Prints one JSON line (rank 0).  --impl reference times the FP64 oracle instead, on
the host cores, over a bounded sample of the same workload.
"""
import argparse
import hashlib
import ctypes as C
import json
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

from paper_2504_01302_b300 import shard, synth  # noqa: E402

METRIC = "joint logL evals/sec and logL+grad evals/sec at 1 B300, at stated FP64-oracle accuracy"
N_SM = 148
# ex2.approx results per clock per SM on B300 (MUFU), measured by a throughput probe
# (profiles/mufu_ffma_rates_b300.md): 32.3-32.8 ex2/clk/SM.
MUFU_EX2_PER_CLK_SM = 32
# FP32 FMA lanes per clock per SM (the same probe measures 3.5-3.8e13 FFMA/s at 2032 MHz)
FFMA_LANES_PER_CLK_SM = 128
# FMA-pipe operations per integrand evaluation in the gradient's JAM kernels: derivative pass
# (exponent 2, prefactor 1, term 1, value and two derivative sums 4), table adjoint (exponent
# 2, weighted term 1, four moment sums 4)
FMA_OPS_PER_EVAL = {"k_jam_fwd_grad": 8, "k_jam_adjoint": 7}
DFMA_PER_CLK_SM = 1.75  # FP64 FMA per clock per SM, measured (profiles/mufu_ffma_rates_b300.md)
DF_OPS_PER_FMA = 12  # FP32 operations of one double-float multiply-add (csrc/k_pixsrc.cu df_fma)


def parse():
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=20)
    p.add_argument("--warmup", type=int, default=3)
    p.add_argument("--impl", default="glad", choices=["glad", "reference"])
    p.add_argument("--workload", type=int, default=1)
    p.add_argument("--grad", action="store_true",
                   help="time only logL + gradient (batch 64); by default both are timed")
    p.add_argument("--no-grad", action="store_true", help="time the forward logL only")
    p.add_argument("--precision", type=int, default=0,
                   help="forward precision mode (glad_set_precision): 0 FP32 bulk, 1 FP64 lensing, "
                        "2 FP64 lensing and pair sum")
    p.add_argument("--batch", type=int, default=0)
    p.add_argument("--no-cpu-baseline", action="store_true")
    p.add_argument("--tuning", default="",
                   help="JAMCODE,EPT: pin the JAM launch shapes instead of autotuning")
    p.add_argument("--graph", type=int, default=-1,
                   help="1: replay the step as a captured CUDA graph (default: on for workload 3)")
    p.add_argument("--pix-path", type=int, default=0,
                   help="evidence evaluation of the pixelated source (glad_set_pix_path): 0 by "
                        "batch size, 1 one CTA per sample, 2 multi-launch")
    p.add_argument("--sph-rule", default="",
                   help="NR,NW,NLOS: rule of the spherically aligned model (default 128,8,32)")
    return p.parse_args()


def ncu_traffic(kernel, w, grad, B):
    """DRAM bytes (read + write) per launch of the timed kernel ``kernel`` from the committed
    ncu summary that captured it on this workload, scaled from the captured batch to B by
    samples (each sample reads its own coefficient table and writes its own accumulators).
    None when no summary matches or when the kernel's sources have changed since the capture:
    each record carries the sha256 of the source files it was built from."""
    here = os.path.dirname(os.path.abspath(__file__))
    pdir = os.path.join(here, "profiles")
    if not os.path.isdir(pdir):
        return None
    for fn in sorted(os.listdir(pdir)):
        if not fn.endswith(".md"):
            continue
        for ln in open(os.path.join(pdir, fn)):
            ln = ln.strip().strip("`")
            if not ln.startswith("traffic-record:"):
                continue
            rec = dict(kv.split("=", 1) for kv in ln.split()[1:])
            if rec["kernel"] != kernel or int(rec["workload"]) != w or int(rec["grad"]) != int(grad):
                continue
            h = hashlib.sha256()
            for f in rec["sources"].split(","):
                with open(os.path.join(here, f), "rb") as fh:
                    h.update(fh.read())
            if h.hexdigest() != rec["sha256"]:
                return None
            return int(rec["dram_bytes"]) * B / int(rec["batch"])
    return None


def workload_name(w, grad, B):
    names = {0: "w0: 64^2 SIE+shear, 10+10 MGE, 32^2 sky, GL32, 20 annuli",
             1: "RXJ1131-scale: 200^2 x2ss, 21^2 PSF, EPL+shear+SIS, 2 lens-light + source Sersic, "
                "JAM 20+2x10+BH, 60^2 sky x4ss, GL32, 50 bins, 4 images",
             3: "8 uneven systems (64..256 px, ss 1-3, 8-30 Gaussians, 20-120 bins, GL 24-64)",
             4: "IFU-scale: 400^2 x3ss, 31^2 PSF, EPL+shear+2 SIS, JAM 40+2x20+BH, 128^2 sky x4, "
                "GL64, 400 bins",
             5: "RXJ1131-scale with the spherically aligned Jeans model (Eqs. J1/J2): 200^2 x2ss, "
                "21^2 PSF, EPL+shear+SIS, JAM 20+2x10+BH, polar grid 128x8, 32 LOS nodes, "
                "60^2 sky x4ss, 50 bins",
             6: "IFU-scale with the spherically aligned Jeans model (Eqs. J1/J2): 400^2 x3ss, "
                "31^2 PSF, EPL+shear+2 SIS, JAM 40+2x20+BH, polar grid 128x8, 32 LOS nodes, "
                "128^2 sky x4, GL64, 400 bins",
             7: "RXJ1131-scale EPL class with the internal mass sheet (dPIE, 40 Gaussians) and "
                "sampled D_d, D_dt,int: 200^2 x2ss, 21^2 PSF, EPL+shear+SIS, JAM 20+40+2x10+BH, "
                "60^2 sky x4ss, GL32, 50 bins",
             8: "RXJ1131-scale composite class (2 Chameleons x Upsilon, eNFW halo as 44 CSEs, BH) "
                "with the dPIE sheet and sampled D_d, D_dt,int (the paper's joint model): 200^2 "
                "x2ss, 21^2 PSF, +shear+SIS, JAM 2x10 tracer x (20 baryon + 20 halo + 40 sheet + BH) "
                "mass, 60^2 sky x4ss, GL32, 50 bins",
             9: "RXJ1131-scale with the pixelated source (Sect. 3.1.1): 200^2 x2ss, 21^2 PSF, "
                "EPL+shear+SIS, 30x30 source grid (N_s = 900), arcs in 0.9-2.5 arcsec (N_d = 6840), "
                "evidence maximised over ln lambda (FP64 Cholesky per evaluation), JAM 20+2x10+BH, "
                "60^2 sky x4ss, GL32, 50 bins",
             10: "Table 3's extended-image timing configuration: RXJ1131-scale composite class "
                 "(2 Chameleons x Upsilon, eNFW halo, BH, dPIE sheet, distance mode 1) with a 64x64 "
                 "source grid (N_s = 4096), arcs in 0.8-2.95 arcsec (N_d = 10148), evidence "
                 "maximised over ln lambda, JAM 2x10 tracer x (20+20+40+BH) mass, 60^2 sky x4ss"}
    n = names.get(w, str(w)) + f"; B={B}"
    if grad:
        n += " (forward + gradient)"
    return n


SPH_NODES = 64  # characteristic nodes per polar grid point of the spherically aligned model


def sph_exp2_counts(systems, sid_np, B, kernel):
    """Algorithmic work of one launch of `kernel` over the batch: for the pair sum and its
    passes, (sky sub-sample, table entry) integrand evaluations (one ex2 each); for the
    spherically aligned model, its integrand exponentials: per polar grid point
    64 x (mass Gaussians x n_gl + tracer Gaussians) along the characteristic plus the same
    at the point itself; per sky sub-sample n_los x (tracer Gaussians + 1) along the line of
    sight plus the tracer surface brightness."""
    n = 0
    for b in range(B):
        s = systems[sid_np[b]]
        nl = sum(s["n_mge_light"])
        nm = s["n_mge_mass"] + (1 if s["has_bh"] else 0)
        nsub = (s["kx"] * s["kss"]) * (s["ky"] * s["kss"])
        if kernel == "k_sph_coef+k_sph_grid":
            n += s["sph_nr"] * s["sph_nw"] * (SPH_NODES + 1) * (nm * s["n_gl"] + nl)
        elif kernel == "k_sph_los":
            n += nsub * (s["sph_nlos"] * (nl + 1) + nl)
        elif kernel == "k_sph_adjoint":
            # line of sight again (one ex2 per node and tracer Gaussian, one per node for e^tau);
            # per grid point, the node sums, the tracer pass and the entry pass over 64 nodes,
            # and the point itself: 130 x (mass x u nodes + tracer)
            n += nsub * s["sph_nlos"] * (nl + 1) + s["sph_nr"] * s["sph_nw"] * 130 * (nm * s["n_gl"] + nl)
        else:
            n += nsub * nl * nm * s["n_gl"]
    if kernel == "k_sph_coef+k_sph_grid":
        return n, f"{n} exponentials per launch (grid points x 65 x (mass x u nodes + tracer))"
    if kernel == "k_sph_los":
        return n, f"{n} exponentials per launch (sky sub-samples x (n_los x (tracer + 1) + tracer))"
    if kernel == "k_sph_adjoint":
        return n, (f"{n} exponentials per launch (sky sub-samples x n_los x (tracer + 1) + grid "
                   f"points x 130 x (mass x u nodes + tracer))")
    return n, f"{n} JAM integrand evaluations per launch (sky sub-samples x table entries)"


def bench_systems(w):
    """Fixed geometry from the seeded generators; data filled in later."""
    bases, B = synth.workload_systems(w)
    out = []
    for b in bases:
        s = dict(b)
        # quasar images on a ring of the Einstein radius (theta[0] of the composite class is the
        # halo's kappa_s, not an Einstein radius)
        s["img_xy"] = synth.ring_images(1.5 if w == 0 else 1.65, s["qso_beta"])
        s["data"] = np.zeros((s["ny"], s["nx"]), np.float32)
        s["v_obs"] = np.ones(s["n_bins"], np.float32)
        s["v_sig"] = np.ones(s["n_bins"], np.float32)
        s["dt_obs"] = np.array([-8.0, 3.5, -12.7, 5.0, 2.0, 1.0, 1.0][:len(s["img_xy"]) - 1])
        s["dt_sig"] = np.full(len(s["img_xy"]) - 1, 0.5)
        out.append(s)
    return out, B


def bench_truth(w, systems):
    if int(systems[0].get("mass_class", 0)) == 1:
        return synth.theta_truth_composite()
    return synth.theta_truth(0 if w == 0 else 1)


def fill_data_with_gpu_model(systems, w, torch, GladContext):
    # the data come from the Sersic source; pixelated-source systems then fit them
    ctx = GladContext([dict(s, src_pix=0) for s in systems])
    truth = torch.as_tensor(bench_truth(w, systems), device="cuda")
    for i, s in enumerate(systems):
        nz = synth.noise_draws(s, 1000 * w + i + 500)
        img = ctx.model_image(truth, i).cpu().numpy().astype(np.float64)
        v = ctx.vrms(truth, i).cpu().numpy().astype(np.float64)
        s["data"] = (img + np.asarray(s["sigma"], np.float64) * nz["img"]).astype(np.float32)
        s["v_sig"] = (0.02 * v).astype(np.float32)
        s["v_obs"] = (v + 0.02 * v * nz["kin"]).astype(np.float32)
    ctx.close()
    return systems


class ClockSampler:
    """nvidia-smi samples of the SM clock and throttle reasons during the timed region."""

    NAMES = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]

    def __init__(self, index):
        self.index = index
        self.rows = []
        self.proc = None

    def __enter__(self):
        q = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.hw_slowdown,"
             "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
             "clocks_event_reasons.sw_power_cap")
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), f"--query-gpu={q}",
                 "--format=csv,noheader,nounits", "-lms", "100"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.th = threading.Thread(target=self._read, daemon=True)
            self.th.start()
        except Exception:
            self.proc = None
        time.sleep(0.3)
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.rows.append([x.strip() for x in line.split(",")])

    def __exit__(self, *a):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(2)
            except Exception:
                self.proc.kill()

    def summary(self):
        sm, mx, reasons = [], None, set()
        for r in self.rows:
            try:
                sm.append(float(r[0]))
                mx = float(r[1])
                for n, v in zip(self.NAMES, r[3:7]):
                    if "Active" in v and "Not" not in v:
                        reasons.add(n)
            except (ValueError, IndexError):
                pass
        loaded = [x for x in sm if x > 0.5 * (mx or 1)] or sm
        return {"sm_mhz": statistics.median(loaded) if loaded else None, "sm_max_mhz": mx,
                "reasons": sorted(reasons), "samples": len(sm)}


def _oracle_eval(s, th):
    sys.path.insert(0, ROOT)
    from oracle import model
    return model.loglike(th, s)


def pix_ns_max(systems):
    return max((int(np.prod(s["spx_n"])) for s in systems if s.get("src_pix", 0)), default=0)


def cpu_baseline(systems, thetas, sids):
    """The FP64 oracle, as it stands, over a bounded sample of the workload on all host cores."""
    import multiprocessing as mp
    cores = os.cpu_count() or 1
    n = cores
    t0 = time.time()
    with mp.get_context("spawn").Pool(cores) as pool:
        res = pool.starmap(_oracle_eval, [(systems[sids[i % len(sids)]], thetas[i % len(thetas)])
                                          for i in range(n)])
    dt = time.time() - t0
    return {"value": n / dt, "unit": "logL/s", "cores": cores, "kind": "oracle",
            "sample": f"{n} samples of the same workload, one per core (spawn pool), {dt:.1f} s wall",
            "finite": int(sum(np.isfinite(res)))}


def run_reference(args):
    """The oracle as the reference arm: host cores, bounded sample per step."""
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    from oracle import model
    w = args.workload
    systems, B = bench_systems(w)
    for i, s in enumerate(systems):
        truth = bench_truth(w, systems)
        s.update(model.build_system(s, truth, synth.noise_draws(s, 1000 * w + i + 500)))
    B = args.batch or (64 if args.grad else B)
    th, sid = synth.workload_thetas(w, B, len(systems))
    import multiprocessing as mp
    cores = os.cpu_count() or 1
    per_step = cores
    times = []
    with mp.get_context("spawn").Pool(cores) as pool:
        for step in range(args.warmup + args.steps):
            idx = [(step * per_step + i) % B for i in range(per_step)]
            t0 = time.time()
            pool.starmap(_oracle_eval, [(systems[sid[i]], th[i]) for i in idx])
            if step >= args.warmup:
                times.append(time.time() - t0)
    T = sum(times)
    val = per_step * len(times) / T
    unit = "logL/s"
    line = {"impl": "reference", "metric": METRIC, "value": val, "unit": unit, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1000 * T / len(times),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic",
            "config": {"workload": workload_name(w, False, B), "samples_per_step": per_step},
            "cpu_baseline": {"value": val, "unit": unit, "cores": cores, "kind": "oracle",
                             "sample": f"{per_step} samples per step, one per host core"},
            "e2e": {"value": val, "unit": unit, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def names_idx(name, lib, nk):
    for i in range(nk):
        if lib.glad_kernel_name(i).decode() == name:
            return i
    raise KeyError(name)


def measure(args, ctx, lib, systems, th_np, sid_np, B, grad_mode, world, rank, local, torch, dist):
    """Time K steps of glad_loglike (or glad_loglike_grad) on this rank's B samples.
    Returns the pieces of the JSON line: device-resident rate, end-to-end rate through the C
    ABI with pinned host buffers, the one-sample-per-call form, per-kernel times from
    separate profiled steps with the two branches serialised, and the roofline of the
    dominant kernel."""
    from paper_2504_01302_b300 import _lib
    w = args.workload
    theta = torch.as_tensor(th_np, device="cuda")
    sid = torch.as_tensor(sid_np, device="cuda")
    logL = torch.empty(B, dtype=torch.float64, device="cuda")
    status = torch.empty(B, dtype=torch.int32, device="cuda")
    grad = torch.empty(B, synth.N_THETA, dtype=torch.float64, device="cuda")
    stream = torch.cuda.current_stream()
    P = lambda t: C.c_void_p(t.data_ptr())

    def step():
        # the stream current at call time: torch.cuda.graph captures on its own stream
        hs = C.c_void_p(torch.cuda.current_stream().cuda_stream)
        if grad_mode:
            rc = lib.glad_loglike_grad(ctx.handle, P(sid), P(theta), B, P(logL), P(grad), P(status),
                                       None, hs)
        else:
            rc = lib.glad_loglike(ctx.handle, P(sid), P(theta), B, P(logL), P(status), None, hs)
        _lib.check(rc, "step")

    ctx.set_precision(0 if grad_mode else args.precision)
    ctx.set_pix_path(args.pix_path)
    # launch shapes picked by the library's autotuner on this batch (untimed), or pinned
    if args.tuning:
        jc, ept = (int(v) for v in args.tuning.split(","))
        ctx.set_tuning(jc, ept)
        tuning = {"jam_pts": jc, "adj_ept": ept}
    else:
        tuning = ctx.autotune(theta, sid, with_grad=grad_mode)
    # L2 flush buffer (256 MB > 126 MB L2), written before each timed step, outside its events
    flush = torch.empty(64 * 1024 * 1024, dtype=torch.float32, device="cuda")
    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    n_valid = int((status == 0).sum())

    # ---- device-resident timing: K steps, events on the launching stream, no profiling
    use_graph = args.graph == 1 or (args.graph == -1 and w == 3)
    graph = None
    if use_graph:
        # the whole step (every kernel of the path) captured once and replayed
        graph = torch.cuda.CUDAGraph()
        with torch.cuda.graph(graph):
            step()
        torch.cuda.synchronize()
        logL.fill_(0.0)
        graph.replay()
        torch.cuda.synchronize()
        # the replay must reproduce the eager step's results
        assert int((status == 0).sum()) == n_valid and bool(torch.isfinite(logL[status == 0]).all())
    lib.glad_profile(ctx.handle, 0)
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
          for _ in range(args.steps)]
    with ClockSampler(local) as clk:
        for k in range(args.steps):
            flush.fill_(float(k))
            ev[k][0].record(stream)
            if use_graph:
                graph.replay()
            else:
                step()
            ev[k][1].record(stream)
        torch.cuda.synchronize()
    t_ms = sum(a.elapsed_time(b) for a, b in ev)
    if world > 1:
        t_ms = shard.max_over_ranks(t_ms, dist, "cuda")
        dist.barrier()
    value = world * B * args.steps / (t_ms / 1000.0)

    # ---- per-kernel times from separate profiled steps (not timed above): both branches on
    # one stream, so each event pair times its kernel alone
    nk = lib.glad_kernel_times(ctx.handle, 0, None, None)
    kms = (C.c_double * nk)()
    kl = (C.c_int * nk)()
    prof_steps = 3
    lib.glad_profile(ctx.handle, 2)
    lib.glad_pix_launches(ctx.handle)  # reset: the pixelated source's launches vary with its search
    for k in range(prof_steps):
        flush.fill_(float(k))
        step()
    torch.cuda.synchronize()
    pix_launches = int(lib.glad_pix_launches(ctx.handle))
    lib.glad_profile(ctx.handle, 0)
    lib.glad_kernel_times(ctx.handle, nk, kms, kl)

    # ---- end to end through the public API with pinned host buffers
    th_h = torch.as_tensor(th_np).pin_memory()
    sid_h = torch.as_tensor(sid_np).pin_memory()
    out_h = torch.empty(B, dtype=torch.float64).pin_memory()
    st_h = torch.empty(B, dtype=torch.int32).pin_memory()
    gr_h = torch.empty(B, synth.N_THETA, dtype=torch.float64).pin_memory()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for k in range(args.steps):
        theta.copy_(th_h, non_blocking=True)
        sid.copy_(sid_h, non_blocking=True)
        step()
        out_h.copy_(logL, non_blocking=True)
        st_h.copy_(status, non_blocking=True)
        if grad_mode:
            gr_h.copy_(grad, non_blocking=True)
    e1.record(stream)
    torch.cuda.synchronize()
    e2e_ms = e0.elapsed_time(e1)
    if world > 1:
        e2e_ms = shard.max_over_ranks(e2e_ms, dist, "cuda")
    h2d = th_h.numel() * 8 + sid_h.numel() * 4
    d2h = out_h.numel() * 8 + st_h.numel() * 4 + (gr_h.numel() * 8 if grad_mode else 0)

    # ---- the plain form: the same kernels called once per sample (B = 1), no graph,
    # on the first n_plain samples of the batch, L2 not flushed between calls
    n_plain = min(B, 4 if any(s.get("src_pix", 0) for s in systems) else 32)

    def plain_call(b):
        hs = C.c_void_p(stream.cuda_stream)
        if grad_mode:
            rc = lib.glad_loglike_grad(ctx.handle, P(sid[b:b + 1]), P(theta[b:b + 1]), 1,
                                       P(logL[b:b + 1]), P(grad[b:b + 1]), P(status[b:b + 1]),
                                       None, hs)
        else:
            rc = lib.glad_loglike(ctx.handle, P(sid[b:b + 1]), P(theta[b:b + 1]), 1,
                                  P(logL[b:b + 1]), P(status[b:b + 1]), None, hs)
        _lib.check(rc, "plain step")

    for b in range(min(n_plain, 3)):
        plain_call(b)
    torch.cuda.synchronize()
    p0, p1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    p0.record(stream)
    for b in range(n_plain):
        plain_call(b)
    p1.record(stream)
    torch.cuda.synchronize()
    plain_ms = p0.elapsed_time(p1)

    extra = kl[names_idx("k_image+k_conv", lib, nk)] + kl[names_idx("k_grad_lens", lib, nk)] + \
        kl[names_idx("k_sph_coef+k_sph_grid", lib, nk)] + 2 * kl[names_idx("k_sph_adjoint", lib, nk)] + \
        (kl[names_idx("k_jam", lib, nk)] if (tuning["jam_pts"] // 100000) % 10 == 1 else 0) + \
        pix_launches - kl[names_idx("k_pix_operator", lib, nk)] - kl[names_idx("k_pix_evidence", lib, nk)]
    launches_per_step = (int(sum(kl[i] for i in range(nk))) + int(extra)) // prof_steps
    if grad_mode:
        launches_per_step += 2  # k_kin_adj and k_grad_zero_invalid run untimed by the profiler
    # integrand evaluations the JAM kernels actually execute per step (exact and negligible
    # terms skipped), from one more untimed full-batch step
    if any(s.get("src_pix", 0) for s in systems):
        ctx.pix_factorizations()  # reset the count: the next step alone is counted
    step()
    n_exec = {"k_jam": ctx.jam_evaluations(), "k_jam_fwd_grad": ctx.jam_evaluations(),
              "k_jam_adjoint": ctx.jam_evaluations(adjoint=True)}
    n_fac = ctx.pix_factorizations() if any(s.get("src_pix", 0) for s in systems) else 0
    # ---- roofline of the dominant kernel (the JAM pair sum, its derivative pass, the table
    # adjoint or a kernel of the spherically aligned model, whichever takes longest per step)
    names = [lib.glad_kernel_name(i).decode() for i in range(nk)]
    per_kernel = {names[i]: kms[i] / max(kl[i], 1) for i in range(nk) if kl[i]}
    jam_name = max((n for n in ("k_jam", "k_jam_fwd_grad", "k_jam_adjoint", "k_sph_coef+k_sph_grid",
                                "k_sph_los", "k_sph_adjoint", "k_pix_evidence") if n in per_kernel),
                   key=lambda n: per_kernel[n])
    jam_ms = per_kernel[jam_name]
    if jam_name == "k_pix_evidence":
        # FP64 flops of the evidence evaluations: per factorisation of F + lambda C (N_s^2)
        # N_s^3 / 3 for the Cholesky, N_s^2 for y = L^-1 D, N_s^2 for assembling F + lambda C
        ns = next(int(np.prod(systems[k]["spx_n"])) for k in sid_np if systems[k].get("src_pix", 0))
        per = ns ** 3 / 3.0 + 2.0 * ns ** 2
        evals = n_fac * per
        units = (f"{evals:.4g} FP64 flops per launch: {n_fac} factorisations of F + lambda C "
                 f"(N_s = {ns}) x (N_s^3/3 + 2 N_s^2)")
        n_exec["k_pix_evidence"] = evals
    else:
        evals, units = sph_exp2_counts(systems, sid_np, B, jam_name)
    # no terms are skipped in the spherically aligned kernels
    n_exec["k_sph_coef+k_sph_grid"] = n_exec["k_sph_los"] = n_exec["k_sph_adjoint"] = evals
    clocks = clk.summary()
    sm_max = clocks["sm_max_mhz"] or 2032.0
    jam_form = tuning["jam_pts"] // 1000000
    if jam_name == "k_pix_evidence":
        # the factorisation's multiply-adds run in double-float on the FP32 pipe, 12 FP32
        # operations each (the GPU's native FP64 rate, 1.75 DFMA/clk/SM, is 6x lower)
        peak = N_SM * FFMA_LANES_PER_CLK_SM / DF_OPS_PER_FMA * 2 * sm_max * 1e6 / 1e12
        peak_unit = "TFLOP/s"
        peak_basis = (f"{N_SM} SM x {FFMA_LANES_PER_CLK_SM} FP32 lanes/clk/SM / {DF_OPS_PER_FMA} "
                      f"FP32 operations per double-float multiply-add x 2 flops x {sm_max:.0f} MHz "
                      f"(FP64-equivalent flops; native FP64: {N_SM} SM x {DFMA_PER_CLK_SM} DFMA/clk "
                      f"= {N_SM * DFMA_PER_CLK_SM * 2 * sm_max * 1e6 / 1e12:.2f} TFLOP/s)")
    elif jam_name == "k_jam" and jam_form in (1, 3):
        # recurrence forms: per 8 evaluations 15 packed FMA-pipe operations (2 FP32 lanes each)
        # and 4 ex2, so the FMA pipe bounds them
        peak = N_SM * FFMA_LANES_PER_CLK_SM * sm_max * 1e6 / 3.75 / 1e9
        peak_unit = "Geval/s"
        peak_basis = (f"{N_SM} SM x {FFMA_LANES_PER_CLK_SM} FP32 lanes/clk/SM x {sm_max:.0f} MHz "
                      f"/ 3.75 FMA-pipe lane operations per evaluation (recurrence form {jam_form})")
    elif jam_name in ("k_jam", "k_sph_coef+k_sph_grid", "k_sph_los", "k_sph_adjoint"):
        # one ex2 per evaluation; the 4 FMA-pipe operations per evaluation allow the same rate
        peak = N_SM * MUFU_EX2_PER_CLK_SM * sm_max * 1e6 / 1e9
        peak_unit = "Gexp2/s"
        peak_basis = (f"{N_SM} SM x {MUFU_EX2_PER_CLK_SM} ex2/clk/SM (measured, "
                      f"profiles/mufu_ffma_rates_b300.md) x {sm_max:.0f} MHz max SM clock")
    else:
        ops = FMA_OPS_PER_EVAL[jam_name]
        peak = N_SM * FFMA_LANES_PER_CLK_SM * sm_max * 1e6 / ops / 1e9
        peak_unit = "Geval/s"
        peak_basis = (f"{N_SM} SM x {FFMA_LANES_PER_CLK_SM} FP32 lanes/clk/SM x {sm_max:.0f} MHz "
                      f"/ {ops} FMA-pipe operations per evaluation")
    executed = n_exec[jam_name]
    if args.precision == 2 and not grad_mode and jam_name == "k_jam":
        executed = evals  # the FP64 pair sum evaluates every term
    scale = 1e12 if peak_unit == "TFLOP/s" else 1e9
    achieved = executed / (jam_ms / 1000.0) / scale
    achieved_alg = evals / (jam_ms / 1000.0) / scale
    unit = "logL+grad/s" if grad_mode else "logL/s"
    return {
        "value": value, "unit": unit, "ms_per_step": t_ms / args.steps, "batch_per_gpu": B,
        "valid_samples": n_valid, "tuning": tuning, "cuda_graph": bool(use_graph),
        "roofline": {"bound": "alu", "kernel": jam_name, "achieved": achieved, "peak": peak,
                     "unit": peak_unit, "frac": achieved / peak,
                     "achieved_basis": ("FP64 flops of the factorisations the search ran (library "
                                        "counter) / the evidence kernels' CUDA-event time alone"
                                        if jam_name == "k_pix_evidence" else
                                        "integrand evaluations the kernel executes per launch "
                                        "(library counter) / its CUDA-event time alone"),
                     "traffic": ncu_traffic(jam_name, w, grad_mode, B),
                     "traffic_basis": "ncu dram__bytes_read.sum + dram__bytes_write.sum of one "
                                      "small-batch capture, scaled by samples to this batch",
                     "executed_evaluations": executed,
                     "algorithmic_units": units,
                     "algorithmic_evaluations": evals,
                     "algorithmic_frac": achieved_alg / peak,
                     "skip_factor": evals / max(executed, 1),
                     "kernel_ms": jam_ms,
                     "peak_basis": peak_basis},
        "kernels_ms_per_step": per_kernel,
        "kernels_note": f"CUDA-event time per launch unit in {prof_steps} profiled steps outside the "
                        "timed region, with the lensing and dynamics branches serialised on one "
                        "stream (in the timed steps they run concurrently on two streams)",
        "plain_form": {"value": n_plain / (plain_ms / 1000.0), "unit": unit, "samples": n_plain,
                       "form": "one sample per call (B = 1), same kernels, no graph"},
        "e2e": {"value": world * B * args.steps / (e2e_ms / 1000.0), "unit": unit,
                "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h},
        # launches of the library's kernels per timed step (count from the profiled steps:
        # k_image and k_conv are one timed unit, the gradient's lensing unit is k_conv_adj +
        # k_image_grad, the persistent JAM form adds k_worklist)
        "gpu_launches": args.steps * launches_per_step,
        "clocks": clocks,
    }


def main():
    args = parse()
    if args.impl == "reference":
        return run_reference(args)
    import torch
    import torch.distributed as dist
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    from paper_2504_01302_b300 import build as _b
    if not _b.up_to_date() and rank == 0:
        _b.build()
    if world > 1:
        dist.barrier()
    from paper_2504_01302_b300.glad import GladContext

    w = args.workload
    systems, B_w = bench_systems(w)
    if args.sph_rule:
        nr, nw, nl = (int(v) for v in args.sph_rule.split(","))
        for s in systems:
            s.update(sph_nr=nr, sph_nw=nw, sph_nlos=nl)
    systems = fill_data_with_gpu_model(systems, w, torch, GladContext)
    ctx = GladContext(systems)
    lib = ctx.lib

    def batch(grad_mode):
        B = args.batch if args.batch and (grad_mode == args.grad) else (64 if grad_mode else B_w)
        # this rank's share of a global batch of world * B samples (no collective on the data)
        th_np, sid_np = shard.shard(*synth.workload_thetas(w, world * B, len(systems)), rank, world)
        return B, th_np, sid_np

    # the forward line (logL/s); with --grad only the gradient line; by default the gradient
    # (logL+grad/s, batch 64) is measured too and reported in the line's "grad" object
    main_grad = bool(args.grad)
    pix = any(s.get("src_pix", 0) for s in systems)
    if main_grad and pix:
        raise SystemExit("the pixelated source has no gradient (glad_loglike_grad refuses it)")
    B, th_np, sid_np = batch(main_grad)
    m = measure(args, ctx, lib, systems, th_np, sid_np, B, main_grad, world, rank, local, torch, dist)
    g = None
    if not main_grad and not args.no_grad and not pix:
        Bg, thg, sidg = batch(True)
        g = measure(args, ctx, lib, systems, thg, sidg, Bg, True, world, rank, local, torch, dist)
        g["config"] = {"workload": workload_name(w, True, Bg)}

    if rank != 0:
        ctx.close()
        if world > 1:
            dist.barrier()
            dist.destroy_process_group()
        return

    line = {
        "metric": METRIC, "value": m["value"], "unit": m["unit"],
        "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": m["ms_per_step"], "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64" if args.precision == 2 else "f32", "data": "synthetic",
        "config": {"workload": workload_name(w, main_grad, B), "batch_per_gpu": B,
                   "precision": ["f32 bulk; f64 MGE, tables and chi^2 reductions",
                                 "f64 ray shooting, light and PSF; f32 Jeans sums",
                                 "f64 forward pass (ray shooting, light, PSF, pair sum, binning)"]
                                [args.precision],
                   "l2": "flushed (256 MB write) before each timed step",
                   "valid_samples": m["valid_samples"],
                   "tuning": m["tuning"], "cuda_graph": m["cuda_graph"],
                   **({"sph_rule": args.sph_rule} if args.sph_rule else {}),
                   **({"pix_path": ("multi-launch" if args.pix_path != 1
                                    else "one CTA per sample")}
                      if any(s.get("src_pix", 0) for s in systems) else {}),
                   "jam_skipping": "terms that underflow to 0 over a sky tile, and (pair sum and "
                                   "derivative pass) terms whose bounded total over the tile "
                                   "stays below 2^-26 of its smallest sum (checked after the sum)"},
    }
    for k in ("roofline", "kernels_ms_per_step", "kernels_note", "plain_form", "e2e",
              "gpu_launches", "clocks"):
        line[k] = m[k]
    if g is not None:
        line["grad"] = g
    if not args.no_cpu_baseline and world == 1:
        if pix_ns_max(systems) > 1024:
            # the oracle's dense FP64 response and evidence search take minutes per sample here
            line["cpu_baseline"] = {"value": None, "unit": "logL/s", "kind": "oracle",
                                    "sample": "not run: one sample of this grid takes the oracle "
                                              "~5 min on one core (a 4096^2 FP64 factorisation "
                                              "per evaluation of the search)"}
        else:
            line["cpu_baseline"] = cpu_baseline(systems, th_np, sid_np)
    print(json.dumps(line), flush=True)
    ctx.close()
    if world > 1:
        dist.barrier()
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
