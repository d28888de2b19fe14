"""Benchmark of one CheFSI cycle on the bulk-3D-like 8x8x8 workload.

Workload (paper Sec. IV stand-in, synthetic, seed 0): 8x8x8 periodic elements,
27-neighbour block stencil, n_b = 64 (N = 32768), N_s = 4096 states, filter
degree m = 20. One step = one pass of the whole hot path through the public
C ABI: Lanczos bounds -> Chebyshev filter -> Cholesky-QR + Rayleigh-Ritz +
rotation (FP64) -> Fermi occupations -> density blocks.

Metric: Chebyshev-filter TFLOP/s (algorithmic 2 * nnz(H) * N_s * m flops over
the filter's device time) plus seconds per CheFSI cycle, for the mixed-precision
filter and for the plain FP64 path. Inputs (X is 1.07 GB FP64, H 0.45 GB) are
larger than L2, so no flush is needed between steps.

Usage:  python bench.py [--gpus N] [--steps K] [--warmup W] [--prec bf16x3]
        python bench.py --impl reference ...   (the FP64 CPU oracle on a bounded sample)
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
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

WORKLOAD = "bulk3d_8x8x8"
# FP64 peak of the GB300 CUDA cores from the unit counts: 152 SMs x 2 DFMA/clk
# x 2 flop x 2.07 GHz. Only a fallback: the bench measures the rate with the
# library's DFMA probe (dgchefsi_selftest_fp64_rate) and uses that.
F64_PEAK_TFLOPS = 1.259
F64_PEAK = {"tflops": F64_PEAK_TFLOPS, "source": "derived from unit counts and clock (probe not run)"}
SPECTRUM = os.path.join(ROOT, "tests", "golden", "bulk3d_8x8x8_spectrum.txt")
METRIC = "CheFSI filter TFLOP/s + s per CheFSI cycle, mixed vs FP64 at Ritz err<=1e-8"


def filter_flops(H, Ns: int, m: int) -> float:
    """2 * (sum of block sizes of H) * N_s per mat-vec, m mat-vecs (the -cI shift
    and recurrence update are O(N N_s) and not counted)."""
    nnz = int(H.values.shape[0])
    return 2.0 * nnz * Ns * m


def filter_bytes_per_step(H, Ns: int, prec: str) -> float:
    """Algorithmic HBM bytes of one tensor-core filter step: read the operand copy
    of Y_k and the FP32 master of Y_{k-1}, write the FP32 master of Y_{k+1} and
    its operand copies, read the operand copy of H once."""
    N = H.N
    nnz = int(H.values.shape[0])
    if prec == "tf32":
        return 4.0 * N * Ns * 3 + 4.0 * nnz
    if prec == "bf16":
        return 2.0 * N * Ns + 4.0 * N * Ns * 2 + 2.0 * N * Ns + 2.0 * nnz
    if prec == "bf16x3":
        return 2.0 * 2 * N * Ns + 4.0 * N * Ns * 2 + 2.0 * 2 * N * Ns + 2.0 * 2 * nnz
    return 8.0 * N * Ns * 3 + 8.0 * nnz


class ClockSampler:
    """nvidia-smi samples (200 ms) during the timed region."""

    def __init__(self, index):
        self.index = index  # nvidia-smi --id value (the device UUID)
        self.proc = None
        self.lines = []

    def __enter__(self):
        q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.index}", f"--query-gpu={q}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except Exception:
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def __exit__(self, *exc):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()

    def summary(self):
        sm, mx, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            f = [x.strip() for x in ln.split(",")]
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
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": mx,
                "reasons": sorted(reasons), "samples": len(sm)}


def profiled_traffic(prec: str, Ns: int, layout: int = -1, order=None):
    """DRAM bytes per launch of the tensor-core filter step from the committed
    ncu summary, if that summary was taken on the current kernel source (its
    recorded source hash matches) for this precision and, when it records one,
    this unit-shape layout; scaled to N_s (traffic grows in proportion). None
    otherwise."""
    import glob
    import hashlib
    src = os.path.join(ROOT, "paper_1606_03416_gb300", "csrc", "tc_kernel.cuh")
    sha = hashlib.sha1(open(src, "rb").read()).hexdigest()[:12]
    for path in glob.glob(os.path.join(ROOT, "profiles", f"k_filter_step_t?_{prec}_bulk3d_*.md")):
        text = open(path).read()
        if f"source-sha1 (paper_1606_03416_gb300/csrc/tc_kernel.cuh, first 12): {sha}" not in text:
            continue
        if "unit-shape-layout:" in text and f"unit-shape-layout: {layout}" not in text:
            continue
        if "unit-order:" in text and order is not None and f"unit-order: {order}" not in text:
            continue
        for line in text.splitlines():
            key = f"traffic-per-launch-bytes-{prec}-Ns"
            if line.startswith(key):
                ns_ref = int(line[len(key):].split(":")[0])
                return float(line.split(":")[1]) * Ns / ns_ref
    return None


def profiled_gram_traffic(Ns: int):
    """DRAM bytes of one k_gemm_nt_f64 Gram launch from the committed ncu
    summary taken at this N_s on the current FP64 kernel source; else None."""
    import glob
    import hashlib
    src = os.path.join(ROOT, "paper_1606_03416_gb300", "csrc", "f64_kernels.cu")
    sha = hashlib.sha1(open(src, "rb").read()).hexdigest()[:12]
    for path in glob.glob(os.path.join(ROOT, "profiles", "k_gemm_nt_f64_*.md")):
        text = open(path).read()
        if f"source-sha1 (paper_1606_03416_gb300/csrc/f64_kernels.cu, first 12): {sha}" not in text:
            continue
        key = f"traffic-per-launch-bytes-gram-Ns{Ns}:"
        for line in text.splitlines():
            if line.startswith(key):
                return float(line[len(key):])
    return None


def profiled_pairs_traffic(Ns: int, N: int):
    """DRAM bytes of one k_slice_pairs_2sm launch of the Gram-shaped product
    (Ns x Ns, one 4096-long K chunk) from the committed ncu summary taken on the
    current kernel source; else None."""
    import glob
    import hashlib
    src = os.path.join(ROOT, "paper_1606_03416_gb300", "csrc", "pair_gemm.cu")
    sha = hashlib.sha1(open(src, "rb").read()).hexdigest()[:12]
    for path in glob.glob(os.path.join(ROOT, "profiles", "k_slice_pairs_2sm_*.md")):
        text = open(path).read()
        if f"source-sha1 (paper_1606_03416_gb300/csrc/pair_gemm.cu, first 12): {sha}" not in text:
            continue
        key = f"traffic-per-launch-bytes-gram-Ns{Ns}:"
        for line in text.splitlines():
            if line.startswith(key):
                return float(line[len(key):])
    return None


def dist_env():
    from paper_1606_03416_gb300.replicas import rank_info
    return rank_info()


def oracle_sample(Ns_sample: int, m: int, reps: int = 1, threads: int = 1):
    """Time the FP64 oracle's filter on the first Ns_sample states (run in a
    child process with the BLAS thread count fixed, so the core count is
    exact)."""
    code = (
        "import os,sys,time,json\n"
        f"sys.path.insert(0,{ROOT!r})\n"
        "import numpy as np\n"
        "from oracle import chefsi as O\n"
        "from paper_1606_03416_gb300 import inputs as G\n"
        f"cfg=G.CONFIGS[{WORKLOAD!r}]\n"
        "H=G.make_blocks(cfg); Ho=O.DGHamiltonian.from_blocksparse(H)\n"
        f"X=G.make_X(H.N,cfg.Ns,cfg.seed)[:{Ns_sample}].T.copy()\n"
        "lam_lo,lam_hi=-1.5,42.0\n"
        "a=lam_lo+(lam_hi-lam_lo)*cfg.Ns/H.N\n"
        "ts=[]\n"
        f"for _ in range({reps}):\n"
        "    t=time.perf_counter()\n"
        f"    O.chebyshev_filter(Ho,X,{m},a,lam_hi,lam_lo)\n"
        "    ts.append(time.perf_counter()-t)\n"
        "print(json.dumps({'t':ts,'nnz':int(H.values.shape[0])}))\n")
    nt = str(int(threads))
    env = dict(os.environ, OMP_NUM_THREADS=nt, OPENBLAS_NUM_THREADS=nt, MKL_NUM_THREADS=nt)
    out = subprocess.run([sys.executable, "-c", code], capture_output=True, text=True, env=env, timeout=1800)
    if out.returncode != 0:
        raise RuntimeError(out.stderr[-2000:])
    r = json.loads(out.stdout.strip().splitlines()[-1])
    return r["t"], r["nnz"]


def run_reference(args):
    rank, world, _ = dist_env()
    if rank != 0:
        return 0
    from paper_1606_03416_gb300 import inputs as G
    cfg = G.CONFIGS[WORKLOAD]
    sample = args.ref_states
    ts, nnz = oracle_sample(sample, cfg.m, reps=args.warmup + args.steps)
    timed = ts[args.warmup:] if len(ts) > args.warmup else ts
    flops = 2.0 * nnz * sample * cfg.m
    v = flops / statistics.mean(timed) / 1e12
    line = {"impl": "reference", "metric": METRIC, "value": v, "unit": "TFLOP/s", "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * statistics.mean(timed),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic (seeded generator, no dataset)",
            "config": {"workload": WORKLOAD, "N": 32768, "Ns": cfg.Ns, "m": cfg.m, "l2": "inputs larger than L2",
                       "sample": f"filter of the first {sample} of {cfg.Ns} states"},
            "cpu_baseline": {"value": v, "unit": "TFLOP/s", "cores": 1, "kind": "oracle",
                             "sample": f"FP64 NumPy oracle filter (m={cfg.m}) on {sample} of {cfg.Ns} states, "
                                       "one BLAS thread"},
            "e2e": {"value": v, "unit": "TFLOP/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


def run_filter_only(args):
    """Filter alone on a (possibly smaller) copy of the workload: the case the
    ncu captures run on. Prints one JSON line with the mean filter time."""
    import torch
    from paper_1606_03416_gb300 import dgchefsi as D
    from paper_1606_03416_gb300 import inputs as G
    base = G.CONFIGS[args.workload]
    H = G.make_blocks(base)
    cfg = G.scaled_copy(base, Ns=args.ns or G.resolve_sizes(base, H)[0], m=args.m or base.m, name=base.name)
    dev = torch.device("cuda:0")
    X = torch.from_numpy(G.make_X(H.N, cfg.Ns, cfg.seed)).to(dev)
    Y = torch.empty_like(X)
    with D.Context(H) as ctx:
        if args.shape:
            G_, T_, L_ = (int(v) for v in args.shape.split(","))
            ctx.set_tile_shape(args.prec, G_, T_, L_)
        if args.unit_order >= 0 and args.prec != "f64":
            ctx.set_unit_order(args.prec, args.unit_order)
        for _ in range(args.warmup):
            ctx.filter(X, cfg.m, 10.0, 45.0, -2.0, prec=args.prec, Y=Y)
        torch.cuda.synchronize()
        s, e = torch.cuda.Event(True), torch.cuda.Event(True)
        s.record()
        for _ in range(args.steps):
            ctx.filter(X, cfg.m, 10.0, 45.0, -2.0, prec=args.prec, Y=Y)
        e.record()
        torch.cuda.synchronize()
        ms = s.elapsed_time(e) / max(args.steps, 1)
        shape = ctx.tile_shape(args.prec) if args.prec != "f64" else None
        order = ctx.unit_order(args.prec) if args.prec != "f64" else None
    fl = filter_flops(H, cfg.Ns, cfg.m)
    print(json.dumps({"mode": "filter-only", "workload": args.workload, "Ns": cfg.Ns, "m": cfg.m, "prec": args.prec,
                      "ms_per_filter": ms, "filter_tflops": fl / (ms * 1e-3) / 1e12, "unit_shape": shape,
                      "unit_order": order}),
          flush=True)
    return 0


def measure_uneven(dev, precs=("bf16x3", "tf32"), reps=3):
    """The graphene-like 2D sheet with uneven element sizes (24 x 20 elements,
    9-neighbour stencil, n_b ~ U{40..120}, N_s = floor(0.55 N), m = 16): every
    element size runs in one persistent launch per step, the unit shape is
    autotuned, and the whole filter is replayed from a CUDA graph."""
    import torch
    from paper_1606_03416_gb300 import dgchefsi as D
    from paper_1606_03416_gb300 import inputs as G
    cfg = G.CONFIGS["sheet2d_24x20"]
    H = G.make_blocks(cfg)
    Ns, _ = G.resolve_sizes(cfg, H)
    X = torch.from_numpy(G.make_X(H.N, Ns, cfg.seed)).to(dev)
    Y = torch.empty_like(X)
    fl = filter_flops(H, Ns, cfg.m)
    out = {"workload": "sheet2d_24x20", "N": H.N, "Ns": Ns, "m": cfg.m, "nb_range": [int(H.nb.min()), int(H.nb.max())],
           "filter_gflop": fl / 1e9}
    with D.Context(H) as ctx:
        for pr in precs:
            ctx.filter_graph(X, cfg.m, 10.0, 45.0, -2.0, prec=pr, Y=Y)   # tunes, captures
            ts = []
            for _ in range(reps):
                s_, e_ = torch.cuda.Event(True), torch.cuda.Event(True)
                torch.cuda.synchronize()
                s_.record()
                ctx.filter_graph(X, cfg.m, 10.0, 45.0, -2.0, prec=pr, Y=Y)
                e_.record()
                torch.cuda.synchronize()
                ts.append(s_.elapsed_time(e_))
            g_, t_, acc, lay = ctx.tile_shape(pr)
            out[pr] = {"ms_per_filter": min(ts), "tflops": fl / (min(ts) * 1e-3) / 1e12,
                       "unit_shape": {"G": g_, "T": t_, "ACC": acc, "layout": lay}, "graph": True}
        # FP64 variant: the same grouped steps on the DFMA pipe, also from a graph;
        # two steps timed (the whole m = 16 filter takes ~16 s at the FP64 rate)
        m64 = 2
        fl64 = filter_flops(H, Ns, m64)
        ctx.filter_graph(X, m64, 10.0, 45.0, -2.0, prec="f64", Y=Y)
        s_, e_ = torch.cuda.Event(True), torch.cuda.Event(True)
        torch.cuda.synchronize()
        s_.record()
        ctx.filter_graph(X, m64, 10.0, 45.0, -2.0, prec="f64", Y=Y)
        e_.record()
        torch.cuda.synchronize()
        t64 = s_.elapsed_time(e_)
        out["f64"] = {"ms_per_step": t64 / m64, "tflops": fl64 / (t64 * 1e-3) / 1e12,
                      "frac_of_fp64_peak": fl64 / (t64 * 1e-3) / 1e12 / F64_PEAK["tflops"],
                      "steps_timed": m64, "graph": True}
    del X, Y
    torch.cuda.empty_cache()
    return out


def run_adjoint(args):
    """Differentiation workload (12^3 elements, 27-neighbour stencil, n_b = 48,
    N_s = 8192, m = 24): the band-energy gradient of one cycle, with the filter
    in FP64 and in the tensor-core form --prec (FP32 iterates). On a 6^3 copy
    (N_s = 1024) both gradients are compared with central differences of the
    GPU's FP64 energy on 32 random tied block entries (h = 1e-4, plus a sweep
    over h on 8 of them) and along one random symmetric direction of all
    entries; with --adjoint-full one forward + backward is also timed at full
    size (tensor-core form; FP64 too with --adjoint-f64)."""
    import torch
    from paper_1606_03416_gb300 import autograd as A
    from paper_1606_03416_gb300 import dgchefsi as D
    from paper_1606_03416_gb300 import inputs as G
    dev = torch.device("cuda:0")
    base = G.CONFIGS["bulk3d_12x12x12"]
    tc = args.prec if args.prec != "f64" else "bf16x3"
    out = {"mode": "adjoint", "workload": base.name, "tensor_core_precision": tc}

    def bounds_for(ctx, X, v, Ns, N):
        b, tmin = ctx.bounds(v, 10)
        return tmin + (b - tmin) * Ns / N, b, tmin

    def timed(fn):
        s_, e_ = torch.cuda.Event(True), torch.cuda.Event(True)
        s_.record()
        r = fn()
        e_.record()
        torch.cuda.synchronize()
        return r, s_.elapsed_time(e_) / 1e3

    small = G.scaled_copy(base, grid=(6, 6, 6), Ns=1024, name="bulk3d_6x6x6")
    H, X0, v0, Ns, Ne = G.make_problem(small)
    with D.Context(H) as ctx:
        X = torch.from_numpy(X0).to(dev)
        v = torch.from_numpy(v0).to(dev)
        a, b, a0 = bounds_for(ctx, X, v, Ns, H.N)
        (E, _, Hb, Xb), t_grad = timed(lambda: ctx.energy_grad(X, small.m, a, b, a0, Ne, small.kT))
        ctx.energy_grad(X, small.m, a, b, a0, Ne, small.kT, prec=tc)  # tunes the unit shape
        (Et, _, Hbt, Xbt), t_grad_tc = timed(lambda: ctx.energy_grad(X, small.m, a, b, a0, Ne, small.kT, prec=tc))
        mirror = A.mirror_index(H)
        tied = A.tie_symmetric(Hb, mirror).cpu().numpy()
        tied_tc = A.tie_symmetric(Hbt, mirror).cpu().numpy()
        gmax = max(float(np.max(np.abs(tied))), 1e-300)
        rng = np.random.default_rng(0)
        picks = [int(rng.integers(0, H.values.shape[0])) for _ in range(32)]
        vals = torch.from_numpy(H.values.copy()).to(dev)

        def energy_at(vv):
            ctx.set_values(vv)
            return ctx.energy_grad(X, small.m, a, b, a0, Ne, small.kT, grad=False)[0]

        def fd_values(h, idx):
            fds = []
            for i in idx:
                ent = torch.tensor(sorted({i, int(mirror[i])}), device=dev)
                e = []
                for sgn in (1.0, -1.0):
                    vv = vals.clone()
                    vv[ent] += sgn * h
                    e.append(energy_at(vv))
                fds.append((e[0] - e[1]) / (2 * h))
            ctx.set_values(vals)
            return np.array(fds)

        if args.no_fd:
            picks = []
        fd = fd_values(1e-4, picks)
        err64 = np.abs(fd - tied[picks]) / gmax if picks else np.zeros(1)
        errtc = np.abs(fd - tied_tc[picks]) / gmax if picks else np.zeros(1)
        # the same 8 entries at four step sizes: truncation error falls as h^2,
        # rounding noise of the energy grows as 1/h
        sweep = {}
        for h in (() if args.no_fd else (1e-3, 1e-4, 1e-5, 1e-6)):
            f8 = fd_values(h, picks[:8])
            sweep[f"{h:g}"] = {"f64": float(np.max(np.abs(f8 - tied[picks[:8]])) / gmax),
                               tc: float(np.max(np.abs(f8 - tied_tc[picks[:8]])) / gmax)}
        # one random symmetric direction over all entries: E(v +- h d)
        r = np.random.default_rng(1).standard_normal(H.values.shape[0])
        d = torch.from_numpy(0.5 * (r + r[mirror])).to(dev)
        dd64, ddtc = float((Hb * d).sum()), float((Hbt * d).sum())
        direc = {}
        for h in (() if args.no_fd else (1e-3, 1e-4, 1e-5)):
            fdd = (energy_at(vals + h * d) - energy_at(vals - h * d)) / (2 * h)
            direc[f"{h:g}"] = {"fd": fdd, "rel_err_f64": abs(fdd - dd64) / abs(dd64),
                               f"rel_err_{tc}": abs(fdd - ddtc) / abs(dd64)}
        ctx.set_values(vals)
        sliced_small = None
        if args.slices > 0:
            ctx.set_subspace_products("sliced_bf16", args.slices)
            (Es, _, Hbs, Xbs), t_sl = timed(lambda: ctx.energy_grad(X, small.m, a, b, a0, Ne, small.kT, prec=tc))
            ctx.set_subspace_products("f64", args.slices)
            sliced_small = {"energy_rel": abs(Es - Et) / abs(Et),
                            "grad_H_rel_max": float(np.max(np.abs(A.tie_symmetric(Hbs, mirror).cpu().numpy()
                                                                  - tied_tc)) / gmax),
                            "grad_X_rel_max": float((Xbs - Xbt).abs().max() / Xbt.abs().max()),
                            "s_forward_backward": t_sl}
    out["fd_check_6x6x6"] = {
        "N": H.N, "Ns": Ns, "m": small.m, "entries": len(picks), "h": 1e-4,
        "max_rel_err_vs_max_grad": {"f64": float(err64.max()), tc: float(errtc.max())},
        "max_rel_err_by_h_8_entries": sweep,
        "directional_derivative": {"analytic_f64": dd64, f"analytic_{tc}": ddtc, "by_h": direc},
        f"{tc}_vs_f64": {"energy_rel": abs(Et - E) / abs(E),
                         "grad_H_rel_max": float(np.max(np.abs(tied_tc - tied)) / gmax),
                         "grad_X_rel_max": float((Xbt - Xb).abs().max() / Xb.abs().max())},
        "s_forward_backward": {"f64": t_grad, tc: t_grad_tc}}
    if sliced_small:
        out["fd_check_6x6x6"][f"{tc}_sliced_vs_{tc}_f64_products"] = sliced_small
    if args.adjoint_full:
        H, X0, v0, Ns, Ne = G.make_problem(base)
        full = {"N": H.N, "Ns": Ns, "m": base.m, "checkpoint_stride": int(np.ceil(np.sqrt(base.m)))}
        with D.Context(H) as ctx:
            X = torch.from_numpy(X0).to(dev)
            v = torch.from_numpy(v0).to(dev)
            a, b, a0 = bounds_for(ctx, X, v, Ns, H.N)
            forms = [(tc, "f64")] + ([(tc, "sliced")] if args.slices > 0 else []) + \
                ([("f64", "f64")] if args.adjoint_f64 else [])
            ref = None
            for p, prod in forms:
                ctx.set_subspace_products("sliced_bf16" if prod == "sliced" else "f64", max(args.slices, 2))
                (E, _, _, _), t_fwd = timed(lambda: ctx.energy_grad(X, base.m, a, b, a0, Ne, base.kT, grad=False,
                                                                    prec=p))
                (E2, _, Hb, Xb), t_all = timed(lambda: ctx.energy_grad(X, base.m, a, b, a0, Ne, base.kT, prec=p))
                key = p if prod == "f64" else f"{p}/sliced"
                full[key] = {"s_forward": t_fwd, "s_forward_and_backward": t_all, "energy": E,
                             "grad_norm_H": float(Hb.norm()), "grad_norm_X": float(Xb.norm())}
                if p == tc and prod == "f64":
                    ref = (E2, Hb, Xb)
                else:
                    if p == tc and ref is not None:
                        full[key]["vs_f64_products"] = {
                            "energy_rel": abs(E2 - ref[0]) / abs(ref[0]),
                            "grad_H_rel_max": float((Hb - ref[1]).abs().max() / ref[1].abs().max()),
                            "grad_X_rel_max": float((Xb - ref[2]).abs().max() / ref[2].abs().max())}
                        ref = None
                    del Hb, Xb
                torch.cuda.empty_cache()
            ctx.set_subspace_products("f64", max(args.slices, 2))
        out["full_12x12x12"] = full
    print(json.dumps(out), flush=True)
    return 0


def run_gram_only(args):
    """One FP64 Gram S = Y^T Y (k_gemm_nt_f64, lower tiles) of the workload's
    block after one warm-up: the profiling case of the cycle's dominant kernel
    (~2 GB on the device at the bench size)."""
    import torch
    from paper_1606_03416_gb300 import dgchefsi as D
    from paper_1606_03416_gb300 import inputs as G
    dev = torch.device("cuda:0")
    cfg = G.CONFIGS[args.workload]
    H = G.make_blocks(cfg)
    Ns, _ = G.resolve_sizes(cfg, H)
    Ns = args.ns or Ns
    Y = torch.from_numpy(G.make_X(H.N, Ns, cfg.seed)).to(dev)
    S = torch.empty((Ns, Ns), dtype=torch.float64, device=dev)
    with D.Context(H) as ctx:
        ctx.gram(Y, S)
        s_, e_ = torch.cuda.Event(True), torch.cuda.Event(True)
        torch.cuda.synchronize()
        s_.record()
        ctx.gram(Y, S)
        e_.record()
        torch.cuda.synchronize()
    ms = s_.elapsed_time(e_)
    nt = (Ns + 63) // 64
    fl = 2.0 * (nt * (nt + 1) // 2) * 64 * 64 * H.N  # the 64 x 64 tiles on and below the diagonal
    print(json.dumps({"mode": "gram-only", "workload": cfg.name, "Ns": Ns, "N": H.N, "ms": ms,
                      "tflops": fl / (ms * 1e-3) / 1e12}), flush=True)
    return 0


def measure_next_rows(ctx, H, X, Ns, m, prec, dev):
    """Steps around the cycle on the same workload, FP64 on the CUDA cores:
    re-alignment to a perturbed basis (R = 216 sample points per element),
    density blocks on all of H's pattern, and Rayleigh-Ritz under each
    orthonormalisation (one filtered block, the same for all three)."""
    import torch
    from paper_1606_03416_gb300 import inputs as G
    stream = torch.cuda.current_stream()

    def timed(fn, reps=2):
        best, out = 1e30, None
        for _ in range(reps):
            s_, e_ = torch.cuda.Event(True), torch.cuda.Event(True)
            torch.cuda.synchronize()
            s_.record(stream)
            out = fn()
            e_.record(stream)
            torch.cuda.synchronize()
            best = min(best, s_.elapsed_time(e_) / 1e3)
        return best, out

    res = {}
    nb = np.asarray(H.nb)
    R = np.full(nb.shape, 216, dtype=np.int32)
    Vo, Vn = G.make_basis_pair(nb, nb, R, delta=0.05, seed=0)
    Vod, Vnd = torch.from_numpy(G.pack_blocks(Vo)).to(dev), torch.from_numpy(G.pack_blocks(Vn)).to(dev)
    Xn = torch.empty_like(X)
    t, _ = timed(lambda: ctx.realign(X, nb, R, Vod, Vnd, X_new=Xn))
    fl = 2.0 * (float((R.astype(np.int64) * nb * nb).sum()) + Ns * float((nb.astype(np.int64) ** 2).sum()))
    res["realign"] = {"ms": t * 1e3, "gflop": fl / 1e9, "tflops": fl / t / 1e12,
                      "frac_of_fp64_peak": fl / t / 1e12 / F64_PEAK["tflops"], "sample_points_per_element": 216}
    Vod = Vnd = Xn = None
    f = torch.full((Ns,), 0.5, dtype=torch.float64, device=dev)
    t, _ = timed(lambda: ctx.density_pattern(X, f), reps=1)
    fl = 2.0 * float(nnz_of(H)) * Ns
    res["density_pattern"] = {"ms": t * 1e3, "gflop": fl / 1e9, "tflops": fl / t / 1e12,
                              "frac_of_fp64_peak": fl / t / 1e12 / F64_PEAK["tflops"]}
    b, tmin = ctx.bounds(torch.ones(H.N, dtype=torch.float64, device=dev), 10)
    Yf = torch.empty_like(X)
    ctx.filter(X, m, tmin + (b - tmin) * Ns / H.N, b, tmin, prec=prec, Y=Yf)
    Yw = torch.empty_like(X)
    rr = {}
    for mode in ("cholqr", "cholqr2", "shifted_cholqr3"):
        ctx.set_orthonormalisation(mode)
        Yw.copy_(Yf)
        t, _ = timed(lambda: ctx.rayleigh_ritz(Yw), reps=1)
        rr[mode] = t
    ctx.set_orthonormalisation("cholqr")
    res["rayleigh_ritz_s_by_orthonormalisation"] = rr
    return res


def nnz_of(H) -> int:
    nb = np.asarray(H.nb, dtype=np.int64)
    rp, col = np.asarray(H.row_ptr), np.asarray(H.col)
    return int(sum(nb[K] * nb[col[e]] for K in range(len(nb)) for e in range(rp[K], rp[K + 1])))


def measure_sliced(ctx, X_warm, state, cycle, vd, Ns, N, m, Ne, kT, args, dev, bf16_peak):
    """Mixed cycles with the Rayleigh-Ritz products rebuilt from exact BF16
    slices, started from the warm block the timed cycles left; one filtered warm
    block through Rayleigh-Ritz with FP64 and with sliced products (accuracy and
    time); the Gram- and rotation-shaped sliced products against the BF16
    tensor peak (tensor work = slice pairs x 2 M N K)."""
    import torch
    from paper_1606_03416_gb300 import dgchefsi as D
    stream = torch.cuda.current_stream()
    ev = lambda: torch.cuda.Event(enable_timing=True)  # noqa: E731
    s = args.slices
    pairs = s * (s + 1) // 2
    warm_prev = state["prev"]
    out = {"slices": s, "slice_pairs": pairs}
    b, _ = ctx.bounds(vd, 10)
    a, a0 = float(warm_prev.max()), float(warm_prev.min())
    Y1 = torch.empty_like(X_warm)
    ctx.filter(X_warm, m, a, b, a0, prec=args.prec, Y=Y1)
    Y2, Y3 = Y1.clone(), Y1.clone()
    ctx.set_subspace_products("sliced_bf16", s)
    ctx.rayleigh_ritz(Y3)                      # first use: workspace and cuBLAS set-up
    del Y3
    res = {}
    for mode, Yb in (("f64", Y1), ("sliced_bf16", Y2)):
        ctx.set_subspace_products(mode, s)
        s_, e_ = ev(), ev()
        torch.cuda.synchronize()
        s_.record(stream)
        r = ctx.rayleigh_ritz(Yb)
        e_.record(stream)
        torch.cuda.synchronize()
        f, _ = ctx.occupations(r, Ne, kT)
        res[mode] = (r, ctx.density_blocks(Yb, f), s_.elapsed_time(e_) / 1e3)
    scale = max(abs(a0), abs(b))
    out["warm_block_vs_f64_products"] = {
        "ritz_err": float((res["f64"][0] - res["sliced_bf16"][0]).abs().max().item() / scale),
        "density_rel_err": float((res["f64"][1] - res["sliced_bf16"][1]).norm().item() / res["f64"][1].norm().item()),
        "orthonormality": float((Y2 @ Y2.T - torch.eye(Ns, dtype=torch.float64, device=dev)).abs().max().item())}
    out["s_rayleigh_ritz"] = {"f64_products": res["f64"][2], "sliced_products": res["sliced_bf16"][2]}
    del Y1, Y2, res
    # whole mixed cycles with sliced products (when the timed cycles used FP64 products)
    if args.subspace != "sliced":
        ctx.set_subspace_products("sliced_bf16", s)
        state["prev"] = warm_prev
        X, Y = X_warm.clone(), torch.empty_like(X_warm)
        _, X, Y = cycle(args.prec, X, Y)
        n0 = D.launch_count()
        t0, t1 = ev(), ev()
        torch.cuda.synchronize()
        t0.record(stream)
        reps = 3
        for _ in range(reps):
            _, X, Y = cycle(args.prec, X, Y)
        t1.record(stream)
        torch.cuda.synchronize()
        out["s_per_cycle"] = t0.elapsed_time(t1) / 1e3 / reps
        out["gpu_launches_per_cycle"] = (D.launch_count() - n0) / reps
        del X, Y
    # the products alone: Gram shape (N_s x N_s, K = N) and rotation shape (N_s x N, K = N_s)
    S = torch.empty((Ns, Ns), dtype=torch.float64, device=dev)
    W = torch.empty_like(X_warm)
    prods = {}
    for name, fn, mnk in (("gram", lambda: ctx.sliced_gemm(X_warm, X_warm, slices=s, out=S), Ns * Ns * N),
                          ("rotation", lambda: ctx.sliced_gemm(S, X_warm, b_rows=False, slices=s, out=W),
                           Ns * N * Ns)):
        ts = []
        for _ in range(3):
            s_, e_ = ev(), ev()
            torch.cuda.synchronize()
            s_.record(stream)
            fn()
            e_.record(stream)
            torch.cuda.synchronize()
            ts.append(s_.elapsed_time(e_))
        t = statistics.median(ts[1:]) * 1e-3
        tens = pairs * 2.0 * mnk / t / 1e12
        kms, kn = ctx.sliced_timing()   # device time of the slice-pair kernel launches of the last call
        prods[name] = {"ms": t * 1e3, "fp64_equivalent_tflops": 2.0 * mnk / t / 1e12, "tensor_tflops": tens,
                       "bound": "tensor", "peak": bf16_peak, "frac": tens / bf16_peak,
                       "slice_pair_kernel": {"kernel": "k_slice_pairs_2sm", "launches": kn, "ms": kms,
                                             "tensor_tflops": pairs * 2.0 * mnk / (kms * 1e-3) / 1e12,
                                             "frac": pairs * 2.0 * mnk / (kms * 1e-3) / 1e12 / bf16_peak}}
    out["products"] = prods
    ctx.set_subspace_products("f64", s)
    state["prev"] = warm_prev
    return out


def run_sliced_only(args):
    """One FP64 product from BF16 slices of Gram shape (C = A A^T, A: --ns x --k,
    seeded Gaussian), timed after one warm-up call: the case the ncu captures
    of the slice-pair kernel run on."""
    import torch
    from paper_1606_03416_gb300 import dgchefsi as D
    from paper_1606_03416_gb300 import inputs as G
    dev = torch.device("cuda:0")
    Hb = G.make_blocks(G.CONFIGS["tiny_2x2x2"])
    M, K = args.ns or 2048, args.k or 8192
    A = torch.from_numpy(np.random.default_rng(0).standard_normal((M, K))).to(dev)
    C = torch.empty((M, M), dtype=torch.float64, device=dev)
    with D.Context(Hb) as ctx:
        for _ in range(max(args.warmup, 1)):
            ctx.sliced_gemm(A, A, slices=args.slices, out=C)
        torch.cuda.synchronize()
        s_, e_ = torch.cuda.Event(True), torch.cuda.Event(True)
        s_.record()
        for _ in range(args.steps):
            ctx.sliced_gemm(A, A, slices=args.slices, out=C)
        e_.record()
        torch.cuda.synchronize()
        ms = s_.elapsed_time(e_) / max(args.steps, 1)
    pairs = args.slices * (args.slices + 1) // 2
    print(json.dumps({"mode": "sliced-only", "M": M, "K": K, "slices": args.slices, "ms": ms,
                      "tensor_tflops": pairs * 2.0 * M * M * K / (ms * 1e-3) / 1e12}), flush=True)
    return 0


def run_rr_only(args):
    """One Rayleigh-Ritz step (Alg. 1 steps 3-5) on the workload's BF16x3-filtered
    block, with --subspace products, bracketed by cudaProfilerStart/Stop
    (profiling case: ncu --profile-from-start off sees only this call). With
    --rr-cycles K the block is the one filtered after K mixed cycles from the
    random start (a warm step, as in the timed cycles); K = 0: the first block.
    A first call on a copy of the block sets up the workspace outside the bracket."""
    import torch
    from paper_1606_03416_gb300 import dgchefsi as D
    from paper_1606_03416_gb300 import inputs as G
    dev = torch.device("cuda:0")
    cfg = G.CONFIGS[args.workload]
    H, X0, v0, Ns, Ne = G.make_problem(cfg)
    stream = torch.cuda.current_stream()
    with D.Context(H) as ctx:
        ctx.set_subspace_products("sliced_bf16" if args.subspace == "sliced" else "f64", max(args.slices, 2))
        ctx.set_eigensolver(args.eigensolver)
        ctx.set_cholesky(args.cholesky)
        ctx.set_refinement_start(args.start_coupling)
        b, tmin = ctx.bounds(torch.from_numpy(v0).to(dev), 10)
        X = torch.from_numpy(X0).to(dev)
        a, a0 = tmin + (b - tmin) * Ns / H.N, tmin
        prev = None
        for _ in range(args.rr_cycles):
            prev = ctx.cycle(X, cfg.m, Ne, cfg.kT, v0=torch.from_numpy(v0).to(dev), prec="bf16x3",
                             prev_ritz=prev)["ritz"].cpu().numpy()
        if prev is not None:
            a, a0 = float(prev[-1]), float(prev[0])
        Y = ctx.filter(X, cfg.m, a, b, a0, prec="bf16x3")
        ctx.rayleigh_ritz(Y.clone())
        s_, e_ = torch.cuda.Event(True), torch.cuda.Event(True)
        torch.cuda.synchronize()
        torch.cuda.profiler.start()
        s_.record(stream)
        ctx.rayleigh_ritz(Y)
        e_.record(stream)
        torch.cuda.synchronize()
        torch.cuda.profiler.stop()
        eig = ctx.eigensolver_stats()
    print(json.dumps({"mode": "rr_only", "workload": cfg.name, "subspace": args.subspace, "slices": args.slices,
                      "warm_cycles": args.rr_cycles, "cholesky": args.cholesky, "ms": s_.elapsed_time(e_),
                      "eigensolver": eig}), flush=True)
    return 0


def read_spectrum(path):
    """The stored exact eigenvalues (tests/golden format: 'eigenvalues: v v ...')."""
    with open(path) as fh:
        for line in fh:
            if line.startswith("eigenvalues:"):
                return np.array([float(x) for x in line.split(":", 1)[1].split()])
    raise ValueError(f"no eigenvalues in {path}")


def reference_spectrum(cfg, H, nocc, dev):
    """Exact lowest nocc eigenvalues of H, an error metric only (outside every
    timed region): the values the oracle's dense eigensolve wrote to
    tests/golden for the 8x8x8 workload, else a dense FP64 eigensolve of H on
    the GPU (torch.linalg.eigvalsh) for other workloads."""
    import torch
    if cfg.name == "bulk3d_8x8x8" and os.path.exists(SPECTRUM):
        lam = read_spectrum(SPECTRUM)
        if lam.size >= nocc:
            return lam[:nocc], "stored oracle eigenvalues (tests/golden/bulk3d_8x8x8_spectrum.txt)"
    N = H.N
    Hd = torch.zeros((N, N), dtype=torch.float64, device=dev)
    vals = torch.from_numpy(np.asarray(H.values)).to(dev)
    nb, off = np.asarray(H.nb), np.concatenate([[0], np.cumsum(np.asarray(H.nb))])
    rp, col, bo = np.asarray(H.row_ptr), np.asarray(H.col), np.asarray(H.blk_off)
    for K in range(len(nb)):
        for e in range(rp[K], rp[K + 1]):
            Kp = int(col[e])
            n0, n1 = int(nb[K]), int(nb[Kp])
            Hd[off[K]:off[K] + n0, off[Kp]:off[Kp] + n1] = vals[bo[e]:bo[e] + n0 * n1].view(n0, n1)
    lam = torch.linalg.eigvalsh(Hd).cpu().numpy()
    del Hd
    torch.cuda.empty_cache()
    return lam[:nocc], "dense FP64 eigensolve of H on the GPU (torch.linalg.eigvalsh)"


def converge_forms(ctx, X0, vd, Ns, N, m, Ne, kT, forms, max_cycles, lam, slices, dev):
    """From the same random start block, CheFSI cycles of each form until the
    Ritz values of the occupied states (i < N_e/2) agree with the exact
    eigenvalues lam to 1e-8 of max(|a0|, |b|) (the normwise reading of the
    target), or max_cycles. A form is a filter precision, optionally
    "/sliced" for Rayleigh-Ritz products from BF16 slices. Each cycle (Lanczos
    bound, filter, Rayleigh-Ritz, occupations, density blocks) is timed with
    CUDA events. Also reported per cycle: the per-value error
    max_i |dlambda_i| / max(|lambda_i|, 1) (1 = a floor in the units of H)."""
    import torch
    stream = torch.cuda.current_stream()
    nocc = lam.size
    out = {}
    for form in forms:
        prec, _, products = form.partition("/")
        ctx.set_subspace_products("sliced_bf16" if products == "sliced" else "f64", max(slices, 2))
        X = torch.from_numpy(X0).to(dev)
        Y = torch.empty_like(X)
        prev, errs, errs_v, times, reached = None, [], [], [], None
        for c in range(max_cycles):
            e0, e1 = torch.cuda.Event(True), torch.cuda.Event(True)
            e0.record(stream)
            b, tmin = ctx.bounds(vd, 10)
            if prev is None:
                a0, a = tmin, tmin + (b - tmin) * Ns / N
            else:
                a, a0 = float(prev.max()), float(prev.min())
            ctx.filter(X, m, a, b, a0, prec=prec, Y=Y)
            ritz = ctx.rayleigh_ritz(Y)
            f, mu = ctx.occupations(ritz, Ne, kT)
            ctx.density_blocks(Y, f)
            e1.record(stream)
            prev = ritz.cpu().numpy()
            times.append(e0.elapsed_time(e1) / 1e3)
            X, Y = Y, X
            d = np.abs(prev[:nocc] - lam[:nocc])
            errs.append(float(np.max(d) / max(abs(a0), abs(b))))
            errs_v.append(float(np.max(d / np.maximum(np.abs(lam[:nocc]), 1.0))))
            if errs[-1] <= 1e-8:
                reached = c + 1
                break
        out[form] = {"cycles_to_target": reached, "ritz_err_by_cycle": errs,
                     "ritz_err_per_value_by_cycle": errs_v,
                     "s_per_cycle_median": float(np.median(times)),
                     "s_to_target": float(np.sum(times)) if reached else None}
        del X, Y
    ctx.set_subspace_products("f64", max(slices, 2))
    return out


def run_converge(args):
    """Cycles to the 1e-8 target for --forms (default: --prec and f64), printed as one JSON line."""
    import torch
    from paper_1606_03416_gb300 import dgchefsi as D
    from paper_1606_03416_gb300 import inputs as G
    dev = torch.device("cuda:0")
    cfg = G.CONFIGS[args.workload]
    H, X0, v0, Ns, Ne = G.make_problem(cfg)
    N, m, kT = H.N, cfg.m, cfg.kT
    nocc = int(np.ceil(Ne / 2))
    t0 = time.time()
    lam, lam_src = reference_spectrum(cfg, H, nocc, dev)
    out = {"mode": "converge", "workload": cfg.name, "N": N, "Ns": Ns, "m": m, "Ne": Ne,
           "states_compared": nocc, "target": 1e-8, "exact_eigenvalues": lam_src,
           "s_exact_eigenvalues": time.time() - t0}
    with D.Context(H) as ctx:
        vd = torch.from_numpy(v0).to(dev)
        forms = [f for f in args.forms.split(",") if f] if args.forms else [args.prec, "f64"]
        out["forms"] = converge_forms(ctx, X0, vd, Ns, N, m, Ne, kT, forms, args.max_cycles, lam, args.slices, dev)
    g = out["forms"].get("f64")
    for form, f in out["forms"].items():
        if form != "f64" and g and f["s_to_target"] and g["s_to_target"]:
            out.setdefault("speedup_to_target", {})[form] = g["s_to_target"] / f["s_to_target"]
    print(json.dumps(out), flush=True)
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="native", choices=["native", "reference"])
    ap.add_argument("--prec", default="bf16x3", choices=["tf32", "bf16", "bf16x3", "f64"])
    ap.add_argument("--f64-steps", type=int, default=1, help="FP64 cycles timed for the per-cycle comparison")
    ap.add_argument("--ref-states", type=int, default=64, help="states in the oracle sample")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-uneven", action="store_true", help="skip the uneven-n_b 2D sheet measurement")
    ap.add_argument("--no-next-rows", action="store_true",
                    help="skip re-alignment, pattern density and orthonormalisation timings")
    ap.add_argument("--adjoint", action="store_true", help="differentiation workload instead of the cycle")
    ap.add_argument("--adjoint-full", action="store_true", help="with --adjoint: also time the full 12^3 size")
    ap.add_argument("--adjoint-f64", action="store_true", help="with --adjoint-full: time the FP64 gradient too")
    ap.add_argument("--no-fd", action="store_true", help="with --adjoint: skip the finite-difference checks")
    ap.add_argument("--converge", action="store_true",
                    help="cycles to Ritz error <= 1e-8 against a dense eigensolve, mixed and FP64")
    ap.add_argument("--max-cycles", type=int, default=40)
    ap.add_argument("--no-converge", action="store_true",
                    help="skip the cycles-to-1e-8 runs (sliced, mixed and FP64 forms) of the default line")
    ap.add_argument("--converge-cycles", type=int, default=8, help="cycle limit of those runs")
    ap.add_argument("--gram-only", action="store_true", help="time one FP64 Gram (profiling case)")
    ap.add_argument("--rr-only", action="store_true", help="one Rayleigh-Ritz step (profiling case)")
    ap.add_argument("--rr-cycles", type=int, default=0, help="--rr-only: mixed cycles run before the profiled step")
    ap.add_argument("--start-coupling", type=float, default=0.001,
                    help="first-order coupling that puts a row in the refined eigensolve's FP32 start block")
    ap.add_argument("--subspace", default="sliced", choices=["f64", "sliced"],
                    help="Rayleigh-Ritz products of the timed cycles (and of --rr-only)")
    ap.add_argument("--eigensolver", default="auto", choices=["auto", "syevd", "refined"],
                    help="eigensolve of the projected H (auto: refined with sliced products)")
    ap.add_argument("--cholesky", default="auto", choices=["auto", "cusolver", "products"],
                    help="Cholesky factorisation of step 3 (auto: recursive on products with sliced products)")
    ap.add_argument("--slices", type=int, default=10,
                    help="BF16 slices of the sliced Rayleigh-Ritz products measured beside the FP64 ones (0: skip)")
    ap.add_argument("--forms", default="",
                    help="converge: comma list of filter[/sliced] forms (default: --prec and f64)")
    ap.add_argument("--workload", default=WORKLOAD)
    ap.add_argument("--filter-only", action="store_true",
                    help="time only the filter (profiling case); --ns and --m override the workload")
    ap.add_argument("--sliced-only", action="store_true",
                    help="one Gram-shaped product from BF16 slices, --ns x --k (profiling case)")
    ap.add_argument("--k", type=int, default=0)
    ap.add_argument("--ns", type=int, default=0)
    ap.add_argument("--m", type=int, default=0)
    ap.add_argument("--shape", default="", help="filter-only: force the unit shape G,T,layout (default: autotune)")
    ap.add_argument("--unit-order", type=int, default=-1,
                    help="filter-only: state tiles per pass over the element groups (default: autotune)")
    args = ap.parse_args()
    if args.impl == "reference":
        return run_reference(args)
    if args.filter_only:
        return run_filter_only(args)
    if args.adjoint:
        return run_adjoint(args)
    if args.converge:
        return run_converge(args)
    if args.gram_only:
        return run_gram_only(args)
    if args.rr_only:
        return run_rr_only(args)
    if args.sliced_only:
        return run_sliced_only(args)

    import torch
    rank, world, local = dist_env()
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=dev)

    from paper_1606_03416_gb300 import dgchefsi as D
    from paper_1606_03416_gb300 import inputs as G

    cfg = G.CONFIGS[args.workload]
    H, X0, v0, Ns, Ne = G.make_problem(cfg)
    N, m, kT = H.N, cfg.m, cfg.kT
    ctx = D.Context(H)
    Xd = torch.from_numpy(X0).to(dev)
    Yd = torch.empty_like(Xd)
    vd = torch.from_numpy(v0).to(dev)
    stream = torch.cuda.current_stream()
    ev = lambda: torch.cuda.Event(enable_timing=True)  # noqa: E731

    state = {"prev": None}
    sliced_timed = args.subspace == "sliced" and args.prec != "f64" and args.slices > 0
    products = "sliced_bf16" if sliced_timed else "f64"
    ctx.set_subspace_products(products, max(args.slices, 2))
    ctx.set_eigensolver(args.eigensolver)
    ctx.set_cholesky(args.cholesky)
    ctx.set_refinement_start(args.start_coupling)

    def cycle(prec, X, Y, timers=None):
        """One CheFSI cycle via the public API; returns (ritz, new X buffer, spare buffer)."""
        b, tmin = ctx.bounds(vd, 10)
        prev = state["prev"]
        if prev is None:
            a0 = tmin
            a = a0 + (b - a0) * Ns / N
        else:
            a, a0 = float(prev.max()), float(prev.min())
        if timers is not None:
            timers[0].record(stream)
        ctx.filter(X, m, a, b, a0, prec=prec, Y=Y)
        if timers is not None:
            timers[1].record(stream)
        ritz = ctx.rayleigh_ritz(Y)
        f, mu = ctx.occupations(ritz, Ne, kT)
        ctx.density_blocks(Y, f)
        state["prev"] = ritz.cpu().numpy()
        return ritz, Y, X

    def barrier():
        if world > 1:
            torch.distributed.barrier()
        torch.cuda.synchronize()

    # ---- warm-up
    X, Y = Xd, Yd
    for _ in range(args.warmup):
        _, X, Y = cycle(args.prec, X, Y)
    # ---- timed cycles: mixed filter, Rayleigh-Ritz products as configured (default: BF16 slices)
    n0 = D.launch_count()
    fl_t = [(ev(), ev()) for _ in range(args.steps)]
    t0, t1 = ev(), ev()
    uuid = getattr(torch.cuda.get_device_properties(dev), "uuid", None)
    gid = f"GPU-{uuid}" if uuid is not None and not str(uuid).startswith("GPU-") else (str(uuid) if uuid else "0")
    with ClockSampler(gid) as clk:
        barrier()
        torch.cuda.profiler.start()  # a launch-list capture with --profile-from-start off sees the timed cycles
        t0.record(stream)
        eig_cycles = []  # per timed cycle: the eigensolve's start block and steps (host fields, no device work)
        for i in range(args.steps):
            _, X, Y = cycle(args.prec, X, Y, fl_t[i])
            st_ = ctx.eigensolver_stats()
            eig_cycles.append({k: st_[k] for k in ("start_order", "start_solver", "steps", "used", "history",
                                                   "update_slices")})
        t1.record(stream)
        barrier()
        torch.cuda.profiler.stop()
    eig_timed = ctx.eigensolver_stats()  # the last timed cycle's eigensolve
    launches = D.launch_count() - n0
    X_warm = X.clone()  # the block the timed cycles left (later measurements reuse X and Y)
    ms_step = t0.elapsed_time(t1) / args.steps
    ms_filter = statistics.mean(a.elapsed_time(b) for a, b in fl_t)
    from paper_1606_03416_gb300.replicas import max_over_ranks
    ms_step, ms_filter = max_over_ranks([ms_step, ms_filter], device=dev)
    fl = filter_flops(H, Ns, m)
    value = world * fl / (ms_filter * 1e-3) / 1e12
    ctx.set_subspace_products("f64", max(args.slices, 2))

    # ---- FP64 peak of the CUDA cores, measured by the library's DFMA probe (best of 10)
    with ClockSampler(gid) as clk64:
        f64_rate = ctx.fp64_rate(10) / 1e12
    F64_PEAK.update({"tflops": f64_rate, "clocks": clk64.summary(),
                     "source": "measured: dgchefsi_selftest_fp64_rate (8 independent DFMA chains per thread, "
                               "8 CTAs x 256 threads per SM, best of 10, CUDA events)",
                     "derived_from_unit_counts": F64_PEAK_TFLOPS})
    f64_peak = F64_PEAK["tflops"]

    # ---- per-launch time of the filter step kernel: T(m) - T(1) over m-1 launches
    Xs = Xd.clone()
    def time_filter(mm, reps=3):
        s, e = ev(), ev()
        best = []
        for _ in range(reps):
            torch.cuda.synchronize()
            s.record(stream)
            ctx.filter(Xs, mm, 10.0, 45.0, -2.0, prec=args.prec, Y=Yd)
            e.record(stream)
            torch.cuda.synchronize()
            best.append(s.elapsed_time(e))
        return statistics.median(best)
    t_m, t_1 = time_filter(m), time_filter(1)
    ms_launch = (t_m - t_1) / (m - 1)
    step_fl = fl / m
    peaks = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json"))) if os.path.exists(
        os.path.join(ROOT, "MEASURED_PEAKS.json")) else {}
    hbm = float(peaks.get("hbm_gbs", 6800.0))
    bf16_peak = float(peaks.get("bf16_tflops", 1900.0))
    src = "measured (MEASURED_PEAKS.json)" if peaks else "fallback"
    byts = filter_bytes_per_step(H, Ns, args.prec)
    if args.prec == "f64":
        rf = {"bound": "alu", "achieved": step_fl / (ms_launch * 1e-3) / 1e12, "peak": f64_peak,
              "unit": "TFLOP/s"}
    else:
        mult = 3.0 if args.prec == "bf16x3" else 1.0
        tpeak = bf16_peak * (1.1 / 2.25) if args.prec == "tf32" else bf16_peak
        t_tensor = mult * step_fl / (tpeak * 1e12)
        t_hbm = byts / (hbm * 1e9)
        if t_hbm >= t_tensor:
            rf = {"bound": "hbm", "achieved": byts / (ms_launch * 1e-3) / 1e9, "peak": hbm, "unit": "GB/s"}
        else:
            rf = {"bound": "tensor", "achieved": mult * step_fl / (ms_launch * 1e-3) / 1e12, "peak": tpeak,
                  "unit": "TFLOP/s"}
    rf["frac"] = rf["achieved"] / rf["peak"]
    rf["traffic"] = (profiled_traffic(args.prec, Ns, ctx.tile_shape(args.prec)[3], ctx.unit_order(args.prec))
                     if args.prec != "f64" else None)
    rf["algorithmic_bytes"] = byts
    if args.prec == "f64":
        rf["kernel"] = "k_filter_step_f64"
    else:
        g_, t_, acc_, lay_ = ctx.tile_shape(args.prec)
        rf["kernel"] = (("k_filter_step_tn" if lay_ >= 1 else "k_filter_step_tc") + f"<{args.prec}, G={g_}, T={t_}"
                        + (", 64-byte slots>" if lay_ == 2 else ">"))
        rf["unit_order"] = ctx.unit_order(args.prec)
    rf["ms_per_launch"] = ms_launch
    rf["peak_source"] = (F64_PEAK["source"] if args.prec == "f64" else
                         src + (" x 1.1/2.25 (nominal TF32/BF16 ratio)" if args.prec == "tf32" else ""))
    if args.prec == "bf16x3":
        rf["work"] = "three BF16 products per step (hi*hi + lo*hi + hi*lo) counted as tensor work"

    # ---- FP64 Gram kernel of the Rayleigh-Ritz step with FP64 products (k_gemm_nt_f64),
    # timed through dgchefsi_gram, one launch
    S = torch.empty((Ns, Ns), dtype=torch.float64, device=dev)
    gms = []
    for _ in range(3):
        s_, e_ = ev(), ev()
        torch.cuda.synchronize()
        s_.record(stream)
        ctx.gram(Xs, S)
        e_.record(stream)
        torch.cuda.synchronize()
        gms.append(s_.elapsed_time(e_))
    nt = (Ns + 63) // 64
    gram_fl = 2.0 * (nt * (nt + 1) // 2) * 64 * 64 * N
    g_ach = gram_fl / (statistics.median(gms) * 1e-3) / 1e12
    roof_gram = {"bound": "alu", "achieved": g_ach, "peak": f64_peak, "unit": "TFLOP/s",
                 "frac": g_ach / f64_peak, "traffic": profiled_gram_traffic(Ns), "kernel": "k_gemm_nt_f64",
                 "ms_per_launch": statistics.median(gms), "peak_source": F64_PEAK["source"],
                 "role": "FP64 Gram of the Rayleigh-Ritz step with FP64 products (not run by the sliced cycle)"}

    # ---- filter throughput of the other tensor-core precisions (filter alone)
    other = {}
    for pr in ("bf16", "bf16x3", "tf32"):
        if pr == args.prec or args.prec == "f64":
            continue
        ts_ = []
        for _ in range(2):
            s_, e_ = ev(), ev()
            torch.cuda.synchronize()
            s_.record(stream)
            ctx.filter(Xs, m, 10.0, 45.0, -2.0, prec=pr, Y=Yd)
            e_.record(stream)
            torch.cuda.synchronize()
            ts_.append(s_.elapsed_time(e_))
        other[pr] = fl / (min(ts_) * 1e-3) / 1e12

    # ---- end to end: pinned host X -> device, filter, Y -> host
    Xh = torch.from_numpy(X0).pin_memory()
    Yh = torch.empty_like(Xh).pin_memory()
    e2e_ms = []
    for i in range(2):
        s, e = ev(), ev()
        torch.cuda.synchronize()
        s.record(stream)
        Xs.copy_(Xh, non_blocking=True)
        ctx.filter(Xs, m, 10.0, 45.0, -2.0, prec=args.prec, Y=Yd)
        Yh.copy_(Yd, non_blocking=True)
        e.record(stream)
        torch.cuda.synchronize()
        e2e_ms.append(s.elapsed_time(e))
    serial = world * fl / (min(e2e_ms) * 1e-3) / 1e12
    # the public host-buffer call: chunks copied in / filtered / copied out on three streams
    ctx.filter_host(Xh, m, 10.0, 45.0, -2.0, prec=args.prec, Y=Yh)
    host_s = []
    for i in range(3):
        torch.cuda.synchronize()
        t0h = time.perf_counter()
        ctx.filter_host(Xh, m, 10.0, 45.0, -2.0, prec=args.prec, Y=Yh)
        host_s.append(time.perf_counter() - t0h)
    e2e = {"value": world * fl / min(host_s) / 1e12, "unit": "TFLOP/s",
           "h2d_bytes_per_step": int(Xh.numel() * 8), "d2h_bytes_per_step": int(Yh.numel() * 8),
           "ms": 1e3 * min(host_s), "serial_copies_tflops": serial,
           "what": "dgchefsi_filter_host on pinned host blocks (copies overlapped with the filter in five "
                   "chunks, small first and last), host wall clock around the synchronous call; serial_copies_tflops: copy in, "
                   "filter, copy out one after the other"}
    # a whole cycle end to end: the block from pinned host memory, one cycle as timed above
    # (the block the timed cycles left, with their last Ritz values for the bounds), the new
    # block and the Ritz values back to pinned host memory
    ctx.set_subspace_products(products, max(args.slices, 2))
    Rh = torch.empty(Ns, dtype=torch.float64).pin_memory()
    Xwh = X_warm.cpu().pin_memory()
    cyc_ms = []
    warm_prev = state["prev"]
    for i in range(2):
        state["prev"] = warm_prev
        s, e = ev(), ev()
        torch.cuda.synchronize()
        s.record(stream)
        Xs.copy_(Xwh, non_blocking=True)
        r_, Xn_, _ = cycle(args.prec, Xs, Yd)
        Yh.copy_(Xn_, non_blocking=True)
        Rh.copy_(r_, non_blocking=True)
        e.record(stream)
        torch.cuda.synchronize()
        cyc_ms.append(s.elapsed_time(e))
    state["prev"] = warm_prev
    ctx.set_subspace_products("f64", max(args.slices, 2))
    e2e_cycle = {"value": 1e-3 * min(cyc_ms), "unit": "s per CheFSI cycle", "higher_is_better": False,
                 "h2d_bytes_per_step": int(Xh.numel() * 8), "d2h_bytes_per_step": int(Yh.numel() * 8 + Rh.numel() * 8),
                 "what": "pinned host block (the one the timed cycles left) -> device, one cycle through the "
                         "public API (as the timed steps), new block and Ritz values -> pinned host; CUDA events"}
    Xwh = None

    # ---- precision of one mixed cycle against one FP64 cycle (FP64 filter and FP64
    # products) from the same block with the same bounds: cold = the random start
    # block (first-cycle bounds), warm = the block left by the warm-up and timed
    # cycles (bounds from their last Ritz values)
    f64 = {}
    if args.f64_steps > 0 and args.prec != "f64":
        warm_prev = state["prev"]
        b, tmin = ctx.bounds(vd, 10)

        def compare(Xstart, a, a0, timed):
            Xa, Ya = Xstart.clone(), torch.empty_like(Xstart)
            Xb, Yb = Xstart.clone(), torch.empty_like(Xstart)
            s, e = ev(), ev()
            torch.cuda.synchronize()
            s.record(stream)
            ctx.filter(Xa, m, a, b, a0, prec="f64", Y=Ya)
            r64 = ctx.rayleigh_ritz(Ya)
            fo, _ = ctx.occupations(r64, Ne, kT)
            P64 = ctx.density_blocks(Ya, fo)
            e.record(stream)
            torch.cuda.synchronize()
            if timed:
                f64["s_per_cycle"] = s.elapsed_time(e) / 1e3
            ctx.filter(Xb, m, a, b, a0, prec=args.prec, Y=Yb)
            rmx = ctx.rayleigh_ritz(Yb)
            scale = max(abs(a0), abs(b))
            out = {"ritz_err": float((rmx - r64).abs().max().item() / scale)}
            # largest principal angle between the occupied subspaces (sine, by
            # power iteration on R = Xm - X64 (X64^T Xm)) and the density error
            n_occ = int(round(Ne / 2))
            X64o, Xmo = Ya[:n_occ], Yb[:n_occ]          # state-major rows
            R = Xmo - (Xmo @ X64o.T) @ X64o
            v = torch.ones(n_occ, dtype=torch.float64, device=dev)
            for _ in range(30):
                v = R @ (R.T @ v)
                v = v / v.norm()
            out["subspace_sin_max"] = float((R.T @ v).norm().item())  # top singular value of R
            fm, _ = ctx.occupations(rmx, Ne, kT)
            Pmx = ctx.density_blocks(Yb, fm)
            out["density_rel_err"] = float((Pmx - P64).norm().item() / P64.norm().item())
            return out

        f64["cold_first_cycle"] = compare(torch.from_numpy(X0).to(dev), tmin + (b - tmin) * Ns / N, tmin, True)
        f64["warm"] = compare(X_warm, float(warm_prev.max()), float(warm_prev.min()), False)
        f64["warm"]["after_cycles"] = args.warmup + args.steps

    # ---- the Rayleigh-Ritz products from exact BF16 slices on the tensor cores:
    # accuracy against FP64 products on a warm block, products alone against the BF16 peak
    sliced = None
    if args.slices > 0 and args.prec != "f64":
        sliced = measure_sliced(ctx, X_warm, state, cycle, vd, Ns, N, m, Ne, kT, args, dev, bf16_peak)
        if sliced_timed:
            sliced["s_per_cycle"] = ms_step / 1e3

    # ---- cycles to Ritz error <= 1e-8 from the random start block, three forms
    conv = None
    if not args.no_converge and args.prec != "f64":
        nocc = int(np.ceil(Ne / 2))
        lam, lam_src = reference_spectrum(cfg, H, nocc, dev)
        forms = [f"{args.prec}/sliced", args.prec, "f64"]
        conv = {"target": 1e-8, "states_compared": nocc, "exact_eigenvalues": lam_src,
                "ritz_err": "max over occupied states i of |lambda_i - lambda_i^exact| / max(|a0|, |b|)",
                "ritz_err_per_value": "max over occupied states i of |lambda_i - lambda_i^exact| / "
                                      "max(|lambda_i^exact|, 1)",
                "forms": converge_forms(ctx, X0, vd, Ns, N, m, Ne, kT, forms, args.converge_cycles, lam,
                                        args.slices, dev)}
        g = conv["forms"].get("f64")
        for form, fr in conv["forms"].items():
            if form != "f64" and g and fr["s_to_target"] and g["s_to_target"]:
                conv.setdefault("speedup_to_target_vs_f64", {})[form] = g["s_to_target"] / fr["s_to_target"]

    clocks = clk.summary()
    conv_f = conv["forms"] if conv else {}
    line = {
        "metric": METRIC, "value": value, "unit": "TFLOP/s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms_step, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": args.prec, "data": "synthetic (seeded generator, random-init blocks)",
        "config": {"workload": args.workload, "grid": list(cfg.grid), "stencil": cfg.stencil, "nb": cfg.nb, "N": N,
                   "Ns": Ns, "m": m, "Ne": Ne, "kT": kT, "filter": args.prec,
                   "subspace": f"sliced_bf16 ({args.slices} slices)" if sliced_timed else "f64",
                   "l2": "inputs larger than L2 (X 1.07 GB FP64), no flush",
                   "parallelism": "replicas" if world > 1 else "single GPU"},
        "s_per_cycle": {"mixed_sliced_products": (ms_step / 1e3 if sliced_timed else
                                                  (sliced["s_per_cycle"] if sliced else None)),
                        "mixed": (conv_f.get(args.prec, {}).get("s_per_cycle_median") if conv_f else
                                  (None if sliced_timed else ms_step / 1e3)),
                        "f64": (conv_f.get("f64", {}).get("s_per_cycle_median") if conv_f else f64.get("s_per_cycle")),
                        "what": "timed steps: " + ("mixed_sliced_products" if sliced_timed else "mixed")
                                + "; the other forms: median cycle of the convergence runs"},
        "cycles_to_1e-8": {k: v["cycles_to_target"] for k, v in conv_f.items()},
        "s_to_1e-8": {k: v["s_to_target"] for k, v in conv_f.items()},
        "filter_ms": ms_filter,
        "mixed_vs_f64_one_cycle": {k: f64[k] for k in ("cold_first_cycle", "warm") if k in f64},
        "roofline": rf, "roofline_gram_f64": roof_gram, "fp64_peak": F64_PEAK,
        "filter_tflops_other_precisions": other,
        "e2e": e2e, "e2e_cycle": e2e_cycle, "gpu_launches": launches, "clocks": clocks,
        "eigensolver_timed_cycle": eig_timed,
        "eigensolver_timed_cycles": eig_cycles,
    }
    if conv:
        line["converge"] = conv
    if sliced:
        line["sliced_products"] = sliced
        g = sliced["products"]["gram"]["slice_pair_kernel"]
        # the dominant kernel of this library in the timed (sliced) cycle
        line["roofline_slice_pairs"] = {
            "bound": "tensor", "achieved": g["tensor_tflops"], "peak": bf16_peak, "unit": "TFLOP/s",
            "frac": g["frac"], "traffic": profiled_pairs_traffic(Ns, N), "kernel": "k_slice_pairs_2sm",
            "ms_per_launch": g["ms"] / max(g["launches"], 1),
            "work": f"{args.slices * (args.slices + 1) // 2} slice pairs x 2 Ns^2 x 4096 per launch (one K chunk of "
                    "the Gram-shaped product)",
            "peak_source": src}
    if not args.no_next_rows and args.prec != "f64":
        Xn_rows = torch.from_numpy(X0).to(dev)
        line["next_rows"] = measure_next_rows(ctx, H, Xn_rows, Ns, m, args.prec, dev)
        Xn_rows = None
    ctx.close()
    X = Y = Xd = Yd = Xs = Xh = Yh = S = X_warm = None  # free the 8x8x8 buffers before the next workload
    torch.cuda.empty_cache()
    if not args.no_uneven and args.prec != "f64":
        line["batched_uneven"] = measure_uneven(dev)
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        ts, nnz = oracle_sample(args.ref_states, m, reps=1)
        cv = 2.0 * nnz * args.ref_states * m / ts[0] / 1e12
        line["cpu_baseline"] = {"value": cv, "unit": "TFLOP/s", "cores": 1, "kind": "oracle",
                                "sample": f"FP64 NumPy oracle filter (m={m}) on {args.ref_states} of {Ns} states, "
                                          f"one BLAS thread, {ts[0]:.1f} s"}
        ncpu = os.cpu_count() or 1
        ns_all = 4 * args.ref_states
        ts_all, _ = oracle_sample(ns_all, m, reps=1, threads=ncpu)
        line["cpu_baseline_all_cores"] = {
            "value": 2.0 * nnz * ns_all * m / ts_all[0] / 1e12, "unit": "TFLOP/s", "cores": ncpu, "kind": "oracle",
            "sample": f"FP64 NumPy oracle filter (m={m}) on {ns_all} of {Ns} states, {ncpu} BLAS threads, "
                      f"{ts_all[0]:.1f} s"}
    if rank == 0:
        print(json.dumps(line), flush=True)
    if world > 1:
        torch.distributed.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
