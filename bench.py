#!/usr/bin/env python
"""Chebyshev-filter benchmark on one GB300 (or N independent replicas).

Workload (default): the large supercell, a 62-atom divacancy cell of the
diamond-like lattice (a = 16.4 bohr, Z = 14 / 6, 620 electrons), graded 32^3
mesh, p = 6 (7.1 M nodes), hydrogenic 1s-2p enrichment (310 functions), Gamma
point, 360 vectors, Chebyshev degree 50, frozen synthetic V_eff. --config c3:
the 8-atom zincblende cell a = 8.5 bohr, graded 16^3 mesh, p = 6, 40
enrichment functions, Monkhorst-Pack 2x2x1 (4 complex k-points), 64 vectors per
k, degree 30. One step is one pass of the whole hot path in the steady
state of the subspace iteration: build_hamiltonian, then the batched filter of
every k-point in defect form from the Ritz pairs of the previous pass
(p_m(A) Q = Q p_m(Theta) + D_m: R = A Q - Q Theta by one FP64-class product,
the 30 degrees of D_m on the tensor cores, the sum in FP64), FP64-class
Cholesky-QR and Rayleigh-Ritz per k, then occupations, the density and the
band-trace adjoint (both from one evaluation of the fields). The Ritz pairs a step starts from come from a few untimed
passes from random vectors.

value = dense-count filter flops of a step / step time (TFLOP/s), with the
flop count sum_k sum_e 2 n_aug,e^2 N_v c_k per degree (c_k = 4 complex, 1 real).
"""
import argparse
import json
import math
import os
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import workloads as W  # noqa: E402

FP32_PEAK_DERIVED = 152 * 128 * 2 * 2.070e9 / 1e12   # FP32 FMA lanes x 2 flops x max SM clock
FP64_PEAK_DERIVED = 152 * 2 * 2 * 2.070e9 / 1e12     # 2 DFMA / clk / SM on GB300
# FP32-pair multiply-add: 12 FP32 instructions (exact product by FMA, two-sum, low-part update)
PAIR_PEAK_DERIVED = 152 * 128 * 2.070e9 / 12 * 2 / 1e12
FALLBACK_HBM_GBS = 6800.0
# DRAM bytes (read + write) per launch from the ncu captures summarised under profiles/, scaled to the
# bench's launch by the units processed (valid while the kernels are unchanged since the capture)
TRAFFIC_TENSOR = {   # bf16 parts of the split -> DRAM bytes per (k, cell, 64-vector) tile
    2: {"bytes_per_tile": (2.044714e9 + 0.008223e9) / 1728, "source": "profiles/k_cell_mma_tma_c3mid_12cube_p6.md"},
    3: {"bytes_per_tile": (3.064588e9 + 0.008374e9) / 1728, "source": "profiles/k_cell_mma_tma_c3mid_12cube_p6.md"},
}
TRAFFIC_FP64 = None   # {"bytes_per_cell", "source"} from a capture of the current FP64 product kernels
# the FP64-class products in pair mode, real data: DRAM bytes of the sum-factorized kernel per launch
# of 64 columns and single-leaf cell, from the capture of the current kernel on the 16^3 supercell
# (3600 single-leaf cells; eight vectors per CTA there); the refined cells' dense product is not in it.
# Complex data has no capture of the current kernel (the one of the small zincblende cell predates the
# chunk-major enrichment rows), so its traffic is reported as unknown.
TRAFFIC_PAIR = {"sf_bytes_per_cell": (2.167341e9 + 0.736962e9) / 3600,
                "source": ("profiles/fp64_class_product_fields_wide_c5mid_16cube_p6.md: k_cell_apply_sf DRAM bytes "
                           "per single-leaf cell, scaled by the single-leaf cells; the refined cells' dense product "
                           "not included")}


def is_complex(w):
    """k-points other than Gamma need complex arithmetic; a 1x1x1 grid is the Gamma point alone."""
    return tuple(w.kgrid) != (1, 1, 1)


def workload_text(w):
    """The workload as the JSON line names it (both arms): cell, mesh, basis, k-points, vectors."""
    zs = "/".join(str(int(z)) for z in sorted(set(np.asarray(w.Z).tolist()), reverse=True))
    kg = tuple(w.kgrid)
    kt = ("MP %dx%dx%d (%d k, complex)" % (kg[0], kg[1], kg[2], len(w.nv))) if is_complex(w) else "Gamma point (real)"
    nvt = ("%d vectors/k" % w.nv[0]) if len(set(w.nv)) == 1 else ("%d-%d vectors/k" % (min(w.nv), max(w.nv)))
    cell = "zincblende" if w.natoms == 8 else "supercell"
    return ("%s: %s a=%g bohr, %d atoms (Z %s), graded %d^3 cells p=%d, %d enrichment functions, %s, %s, "
            "Chebyshev degree %d"
            % (w.name, cell, w.a, w.natoms, zs, w.ncell, w.p, len(W.ORBITALS_1S_2P) * w.natoms, kt, nvt, w.degree))


def nucleus_cells(w):
    """Cells whose closed box holds a nucleus (periodic images included): the refined cells."""
    xb = W.mesh_breakpoints(w)
    tol = 1e-12 * w.a
    hold = set()
    for R in w.pos:
        per_axis = []
        for d in range(3):
            x = R[d] % w.a
            idx = [i for i in range(w.ncell) for y in (x - w.a, x, x + w.a) if xb[d][i] - tol <= y <= xb[d][i + 1] + tol]
            per_axis.append(sorted(set(idx)))
        for iz in per_axis[2]:
            for iy in per_axis[1]:
                for ix in per_axis[0]:
                    hold.add((iz * w.ncell + iy) * w.ncell + ix)
    return len(hold)


def measured_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        try:
            return json.load(open(p)), "measured"
        except Exception:
            pass
    return {"hbm_gbs": FALLBACK_HBM_GBS}, "fallback"


class ClockSampler:
    """nvidia-smi clock / throttle samples during the timed region."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device):
        self.device = device
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.device), "--query-gpu=" + self.Q,
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except Exception:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            f = [x.strip() for x in ln.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                smax.append(float(f[2]))
            except ValueError:
                continue
            for nm, v in zip(names, f[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        return {"sm_mhz": float(np.median(sm)) if sm else None, "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


def progress(msg, t0=[time.time()]):
    """One line of progress on stderr (the JSON result goes to stdout), with the device memory in use."""
    used = ""
    try:
        import torch
        if torch.cuda.is_available():
            fr, tot = torch.cuda.mem_get_info()
            used = " [%.1f of %.1f GB in use]" % ((tot - fr) / 1e9, tot / 1e9)
    except Exception:
        pass
    print("[bench %7.1f s] %s%s" % (time.time() - t0[0], msg, used), file=sys.stderr, flush=True)


def barrier(world):
    """Barrier over the replicas (no-op for one process)."""
    if world > 1:
        import torch
        torch.distributed.barrier()


def max_over_ranks(x, world, device="cpu"):
    """The largest value of x over all ranks: the timed region ends when the slowest replica does."""
    if world == 1:
        return float(x)
    import torch
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.MAX)
    return float(t.item())


def whole_job_tflops(flops_per_rank, world, ms):
    """Whole-job throughput: the work every replica did, over the slowest replica's time."""
    return world * flops_per_rank / (ms * 1e-3) / 1e12


def dense_filter_flops(ctx_naug, nvs, degree, cplx=True):
    """sum over k of sum_e 2 n_aug,e^2 N_v,k c_k per degree (c_k = 4 complex, 1 real), times the degree."""
    s2 = float(np.sum(np.asarray(ctx_naug, float) ** 2))
    return sum(2.0 * s2 * nv * (4.0 if cplx else 1.0) for nv in nvs) * degree


def kernel_flops_per_launch(naug, nv, cplx=True):
    return 2.0 * float(np.sum(np.asarray(naug, float) ** 2)) * nv * (4.0 if cplx else 1.0)


# ----------------------------------------------------------------------------- GPU arm
def run_ours(args, rank, world):
    import torch
    import paper_2010_09701_gb300 as P

    dev = int(os.environ.get("LOCAL_RANK", 0))
    torch.cuda.set_device(dev)
    w = W.CONFIGS[args.config]()
    t0 = time.time()
    kpts = None
    if args.filter_only:   # profiling aid: the first k-point only
        k_all, _ = W.monkhorst_pack(w.a, w.kgrid)
        kpts = (k_all[:1], np.array([1.0]))
        w.nv = w.nv[:1]
    ctx = P.setup_workload(w, device=dev, kpoints=kpts)
    nh, nO = ctx.ndof()
    n = nh + nO
    nk = ctx.nk
    xyz, qw = ctx.quadrature_points()
    V = W.veff_device(xyz, w.a, w.pos, w.Z, w.sigma, device="cuda")
    cplx = is_complex(w)
    vdt = torch.complex128 if cplx else torch.float64      # FP64-class vectors
    ldt = torch.complex64 if cplx else torch.float32       # low-precision vectors
    dt64 = P.C128 if cplx else P.F64
    dt32 = P.C64 if cplx else P.F32
    bf16x3 = args.split == "bf16x3"
    split = P.STORE_BF16X3 if bf16x3 else P.STORE_BF16X6
    store = P.STORE_F64 | (split if args.tensor else P.STORE_F32)
    pairs = args.f64_products == "pairs"
    if pairs:
        store |= P.STORE_F64PAIR
    # the compact FP64 layout (enrichment strips of single-leaf cells) when the whole FP64 copies
    # would take more than a quarter of the device
    ncells = w.ncell ** 3
    naug = np.array([len(ctx.cell_info(e)) for e in range(ncells)])
    npad = -(-int(naug.max()) // 128) * 128
    full64 = ncells * npad * npad * (16 if cplx else 8) * (2 if pairs else 1) * nk
    dev_bytes = torch.cuda.get_device_properties(dev).total_memory
    compact = args.compact == "on" or (args.compact == "auto" and full64 > dev_bytes / 4)
    if compact:
        store |= P.STORE_COMPACT
    ctx.set_f64_products(P.F64_PAIRS if pairs else P.F64_NATIVE)
    ctx.set_product_shape(args.product_shape)
    if args.filter_only:   # profiling aid: the low-precision matrices (and FP64 ones on request) only
        store = ((split if args.tensor else P.STORE_F32) | (P.STORE_F64 if args.with_fp64 else 0) |
                 (store & P.STORE_COMPACT))
        if args.with_fp64 and pairs:
            store |= P.STORE_F64PAIR
    progress("set up: %d dof, %d points; building (store %d)" % (n, len(qw), store))
    ctx.build_hamiltonian(V, store)
    progress("operator built")
    if args.filter_only:
        ctx.release_workspace()   # the build's scratch is several times the filter's
    nvs = w.nv
    deg = w.degree
    X0 = [torch.tensor(W.random_vectors(n, nvs[ik], complex_=cplx, seed=w.seed + ik), dtype=vdt, device="cuda")
          for ik in range(nk)]
    X = [x.clone() for x in X0]
    # filter bounds: b from a Lanczos run per k; a, a0 below/above the wanted window
    bks = []
    for ik in range(nk):
        v0 = torch.tensor(W.random_vectors(n, 1, complex_=cplx, seed=100 + ik), dtype=vdt, device="cuda")
        bks.append(ctx.upper_bound(ik, v0, 20, P.FILTER_BF16X3 if (args.tensor or args.filter_only) else 0))
    a_lo, a0 = 0.0, -0.5 * float(max(w.Z)) ** 2 - 1.0
    rho = torch.zeros(len(qw), dtype=torch.float64, device="cuda")
    gV = torch.zeros_like(rho)
    setup_s = time.time() - t0
    stream = torch.cuda.current_stream()

    filt_events = []
    phase_ms = {}
    fflags = P.FILTER_LAST_FP64 | (P.FILTER_BF16X3 if args.tensor else 0)
    if args.filter_only:
        X32 = X0[0].to(ldt)
        if args.batched_filter:   # the batched launch on one group of at most 128 vectors, a fixed shape
            ctx.set_filter_shape(args.filter_shape)
            Xg = X32[:, :min(nvs[0], 128)].contiguous()
            for _ in range(args.steps):
                ctx.filter_batched([Xg], deg, [a_lo], [bks[0]], [a0], P.FILTER_BF16X3)
        else:
            for _ in range(args.steps):
                ctx.chebyshev_filter(0, X32, deg, a_lo, bks[0], a0, flags=P.FILTER_BF16X3 if args.tensor else 0)
        if args.with_fp64:   # one FP64 operator application (the FP64 cell product)
            Y64 = torch.empty_like(X0[0])
            ctx.apply_h(0, X0[0], Y64)
        if args.with_density:   # the fields of the filtered vectors (density at the points)
            occ = np.full(nvs[0], 2.0 / nvs[0])
            ctx.density([X0[0]], [occ], rho)
        if args.with_ortho:     # two Cholesky-QR of the FP64 vectors (Gram matrices and rotations)
            for _ in range(2):
                Xq = X0[0].clone()
                ctx.orthonormalize(0, Xq)
        torch.cuda.synchronize()
        return {"filter_only": True, "passes": args.steps, "config": w.name}

    def mark():
        ev = torch.cuda.Event(enable_timing=True)
        ev.record(stream)
        return ev

    batched = args.tensor and not args.per_k_filter
    defect = batched and not args.plain_filter
    tune_ms = None
    if batched:
        # on at most one batched group of vectors per k (wider blocks run as several groups)
        tune_ms = [float(x) for x in ctx.filter_autotune([x[:, :min(x.shape[1], 128)] for x in X0])]

    def subspace_pass(Xs, bnd, theta, resid=False):
        """One pass of the subspace iteration over all k (outside the timed region): the batched
        filter (defect form from the previous Ritz pairs when theta is given), Cholesky-QR,
        Rayleigh-Ritz. Returns Ritz values, residuals and the next pass's bounds."""
        lo = [bd[0] for bd in bnd]
        low = [bd[1] for bd in bnd]
        if theta is None:
            ctx.filter_batched(Xs, deg, lo, bks, low, P.FILTER_BF16X3 | P.FILTER_LAST_FP64)
        else:
            ctx.filter_batched_defect(Xs, deg, lo, bks, low, theta, P.FILTER_BF16X3)
        out = []
        for ik in range(nk):
            ctx.orthonormalize(ik, Xs[ik])
            out.append(ctx.rayleigh_ritz(ik, Xs[ik], resid=True))
        ev = [o[0] for o in out]
        res = [o[1] for o in out]
        # Zhou's bounds for the next pass: a = the largest Ritz value, a0 below the smallest
        return ev, res, [(float(e[-1]), float(e[0]) - 1.0) for e in ev]

    # the state a step starts from: Ritz pairs after a few passes from the random start vectors (the
    # steady state of the subspace iteration inside an SCF loop), untimed
    theta0 = None
    bnd0 = [(a_lo, a0)] * nk
    if defect:
        Xs = [x.clone() for x in X0]
        theta0 = None
        for _ in range(args.init_passes):
            theta0, _res, bnd0 = subspace_pass(Xs, bnd0, theta0)
        for ik in range(nk):
            X0[ik].copy_(Xs[ik])
        del Xs
    lo_k = [bd[0] for bd in bnd0]
    low_k = [bd[1] for bd in bnd0]

    def step(record=False):
        t = [mark()]
        ctx.build_hamiltonian(V, store)
        t.append(mark())
        eigs = []
        ortho_rr = []
        if batched:
            # every k-point in one persistent tensor-core launch per degree (graph-captured)
            for ik in range(nk):
                X[ik].copy_(X0[ik])
            e0 = mark()
            if defect:   # from the Ritz pairs (X0, theta0): p_m(A) X0 = X0 p_m(theta0) + D_m
                ctx.filter_batched_defect(X, deg, lo_k, bks, low_k, theta0, P.FILTER_BF16X3)
            else:
                ctx.filter_batched(X, deg, a_lo, bks, a0, fflags)
            e1 = mark()
            if record:
                filt_events.append((e0, e1))
        for ik in range(nk):
            if not batched:
                X[ik].copy_(X0[ik])
                e0 = mark()
                ctx.chebyshev_filter(ik, X[ik], deg, a_lo, bks[ik], a0, flags=fflags)
                e1 = mark()
                if record:
                    filt_events.append((e0, e1))
            else:
                e0 = e1 = mark()
            ctx.orthonormalize(ik, X[ik])
            e2 = mark()
            eigs.append(ctx.rayleigh_ritz(ik, X[ik]))
            ortho_rr.append((e0, e1, e2, mark()))
        t.append(mark())
        mu, occ, eb = P.occupations(eigs, [1.0 / nk] * nk, w.nelectrons)
        # the density and the band-trace gradient of k = 0 from one evaluation of the fields
        ctx.density_grad(X, occ, rho, 0, gV)
        t.append(mark())
        if record:
            torch.cuda.synchronize()
            phase_ms.clear()
            phase_ms["build_hamiltonian"] = t[0].elapsed_time(t[1])
            phase_ms["filter"] = (filt_events[-1][0].elapsed_time(filt_events[-1][1]) if batched
                                  else sum(a.elapsed_time(b) for a, b, _, _ in ortho_rr))
            phase_ms["orthonormalize"] = sum(b.elapsed_time(c) for _, b, c, _ in ortho_rr)
            phase_ms["rayleigh_ritz"] = sum(c.elapsed_time(d) for _, _, c, d in ortho_rr)
            phase_ms["density_and_band_trace_grad"] = t[2].elapsed_time(t[3])
        return eigs, eb

    progress("start state ready; %d warm-up steps" % args.warmup)
    for _ in range(args.warmup):
        step()
    progress("timed steps")
    torch.cuda.synchronize()
    barrier(world)
    sampler = ClockSampler(dev)
    sampler.start()
    ctx.kernel_timing([dt32])
    torch.cuda.synchronize()
    barrier(world)
    ev0 = torch.cuda.Event(enable_timing=True)
    ev1 = torch.cuda.Event(enable_timing=True)
    launches0 = P.launch_count()
    torch.cuda.nvtx.range_push("timed_steps")   # lets a profiler take the launches of the timed region
    ev0.record(stream)
    for _ in range(args.steps):
        eigs, eb_mixed = step(record=True)
    ev1.record(stream)
    torch.cuda.nvtx.range_pop()
    launches = P.launch_count() - launches0
    torch.cuda.synchronize()
    barrier(world)
    clocks = sampler.stop()
    progress("timed: %.1f ms per step, phases %s" % (ev0.elapsed_time(ev1) / args.steps,
                                                      {k_: round(v_, 1) for k_, v_ in phase_ms.items()}))
    kms, klaunch = ctx.kernel_time()
    ctx.kernel_timing([])
    step_ms = max_over_ranks(ev0.elapsed_time(ev1) / args.steps, world, "cuda")
    filt_ms = [a.elapsed_time(b) for a, b in filt_events]
    flops_step = dense_filter_flops(naug, nvs, deg, cplx)
    value = whole_job_tflops(flops_step, world, step_ms)
    filt_tflops = flops_step / (sum(filt_ms) / args.steps * 1e-3) / 1e12
    # seconds per filter pass of one k-point
    s_per_pass = float(np.mean(filt_ms)) * 1e-3 / (nk if batched else 1)
    # dominant kernel: the FP32 (complex64) cell product
    per_launch_ms = kms / max(klaunch, 1)
    # a batched launch covers every k-point and one group of at most 128 vectors per k
    ngroups = -(-max(nvs) // 128)
    nv_launch = [-(-v // ngroups) for v in nvs] if batched else nvs[:1]
    kflops = sum(kernel_flops_per_launch(naug, v, cplx) for v in nv_launch)
    nparts = 2 if bf16x3 else 3                # bf16 parts per real value of the split matrices
    nprod = 3 if bf16x3 else 6                 # products per element on the tensor cores
    cf = 2 if cplx else 1                      # real planes per matrix entry / reals per vector entry
    kbytes = sum(float(np.sum(naug ** 2)) * 2 * nparts * cf + 2 * float(np.sum(naug)) * v * 4 * cf for v in nv_launch)
    achieved = kflops / (per_launch_ms * 1e-3) / 1e12
    peaks, src = measured_peaks()
    if args.tensor:
        hbm = peaks.get("hbm_gbs", FALLBACK_HBM_GBS)
        ach = kbytes / (per_launch_ms * 1e-3) / 1e9
        roof_low = {"kernel": ("k_cell_mma_tma<%s> (tcgen05 + TMA, BF16x%d)" % ("complex" if cplx else "real", nprod)
                               + (" over all k" if batched else "")),
                    "bound": "hbm", "achieved": ach, "peak": hbm,
                    "unit": "GB/s", "frac": ach / hbm,
                    "traffic": (TRAFFIC_TENSOR[nparts]["bytes_per_tile"] * len(naug) * sum((v + 63) // 64 for v in nv_launch)
                                if (nparts in TRAFFIC_TENSOR and cplx) else None),
                    "traffic_source": (TRAFFIC_TENSOR[nparts]["source"] + " (scaled by tiles)"
                                       if (nparts in TRAFFIC_TENSOR and cplx) else None),
                    "algorithmic_bytes_per_launch": kbytes,
                    "launches": klaunch, "ms_per_launch": per_launch_ms, "peak_source": src,
                    "dense_tflops": achieved,
                    "tensor_frac_bf16": nprod * achieved / peaks.get("bf16_tflops", 1911.8)}
    else:
        roof_low = {"kernel": "k_cell_apply<float,complex>", "bound": "alu", "achieved": achieved,
                    "peak": FP32_PEAK_DERIVED, "unit": "TFLOP/s", "frac": achieved / FP32_PEAK_DERIVED,
                    "traffic": None, "algorithmic_bytes_per_launch": kbytes, "launches": klaunch,
                    "ms_per_launch": per_launch_ms, "peak_source": "derived: 152 SM x 128 FP32 lanes x 2 x 2070 MHz",
                    "hbm_gbs_at_algorithmic_bytes": kbytes / (per_launch_ms * 1e-3) / 1e9}

    # plain FP64 GPU filter pass on k = 0, for the mixed-vs-FP64 comparison
    fp64 = None
    accuracy = None
    fp64_ms_launch = None
    if not args.skip_fp64:
        # one FP64 filter pass (k = 0) from the same start vectors, the FP64 cell product timed live.
        # Blocks wider than 64 vectors go through the FP64 filter in independent chunks of 64 columns:
        # one chunk is timed and the pass time scaled by the chunk count (the columns are independent
        # and every chunk does the same work)
        ctx.set_f64_products(P.F64_NATIVE)
        vslice = min(nvs[0], 64)
        fp64_scale = nvs[0] / vslice
        Xf = X0[0][:, :vslice].clone()
        ctx.chebyshev_filter(0, Xf, 1, a_lo, bks[0], a0)   # warm
        Xf.copy_(X0[0][:, :vslice])
        torch.cuda.synchronize()
        ctx.kernel_timing([dt64])
        f0 = torch.cuda.Event(enable_timing=True)
        f1 = torch.cuda.Event(enable_timing=True)
        f0.record(stream)
        ctx.chebyshev_filter(0, Xf, deg, a_lo, bks[0], a0)
        f1.record(stream)
        torch.cuda.synchronize()
        k64_ms, k64_n = ctx.kernel_time()
        ctx.kernel_timing([])
        del Xf
        fp64_ms_launch = k64_ms / max(k64_n, 1)
        fp64_s = f0.elapsed_time(f1) * 1e-3 * fp64_scale
        # the FP64-class product of the mixed step (FP32 pairs on the single-leaf cells), timed live
        # on the same vectors
        mix_ms_launch = fp64_ms_launch
        if pairs:
            ctx.set_f64_products(P.F64_PAIRS)
            Xs_ = X0[0][:, :vslice].contiguous()
            Yp = torch.empty_like(Xs_)
            ctx.apply_h(0, Xs_, Yp)   # warm
            torch.cuda.synchronize()
            ctx.kernel_timing([dt64])
            for _ in range(3):
                ctx.apply_h(0, Xs_, Yp)
            torch.cuda.synchronize()
            kp_ms, kp_n = ctx.kernel_time()
            ctx.kernel_timing([])
            mix_ms_launch = kp_ms / max(kp_n, 1)
            del Yp
        progress("FP64 filter pass %.2f s" % fp64_s)
        fp64 = {"s_per_pass_k0": fp64_s,
                "tflops": dense_filter_flops(naug, [nvs[0]], deg, cplx) / fp64_s / 1e12,
                "speedup_mixed_vs_fp64": fp64_s / s_per_pass}
        if fp64_scale != 1.0:
            fp64["timed_columns"] = vslice
            fp64["scaled_to_columns"] = nvs[0]

        # accuracy at convergence: the subspace iteration of the step (defect-form mixed filter from the
        # previous Ritz pairs, FP64-class Cholesky-QR and Rayleigh-Ritz, every k) runs from the step's
        # starting state until the largest residual of the occupied states is below the 1e-7 target or
        # stops falling; then one pass with the native FP64 filter (FP64 products, Cholesky-QR and
        # Rayleigh-Ritz) from that subspace is compared with it
        if defect:
            # the step's buffers hold the iteration (every step copies its start from X0 again)
            Xc = X
            for ik in range(nk):
                Xc[ik].copy_(X0[ik])
            theta, bnd = theta0, bnd0
            hist = []
            occ_idx = None
            t_acc = time.time()
            for it in range(args.acc_passes):
                theta, res, bnd = subspace_pass(Xc, bnd, theta)
                _, occ_m, e_m = P.occupations(theta, [1.0 / nk] * nk, w.nelectrons)
                occ_idx = [np.asarray(o) > 1e-8 for o in occ_m]
                hist.append(float(max(np.max(np.asarray(r)[o]) for r, o in zip(res, occ_idx))))
                if len(hist) % 5 == 0:
                    progress("accuracy pass %d: residual %.3e" % (len(hist), hist[-1]))
                if hist[-1] < args.acc_target * 0.1 or time.time() - t_acc > args.acc_seconds:
                    break
                if len(hist) > 25 and hist[-1] > 0.5 * min(hist[:-20]):
                    break   # no longer falling
            acc_s = time.time() - t_acc
            progress("accuracy run: %d passes, residual %.2e" % (len(hist), hist[-1]))
            ev_m = theta
            # one FP64 pass from the converged subspace: native FP64 filter, Cholesky-QR, Rayleigh-Ritz
            ctx.set_f64_products(P.F64_NATIVE)
            ev_d, res_d = [], []
            for ik in range(nk):   # in place: the mixed state is not needed any more
                ctx.chebyshev_filter(ik, Xc[ik], deg, bnd[ik][0], bks[ik], bnd[ik][1])
                ctx.orthonormalize(ik, Xc[ik])
                e_, r_ = ctx.rayleigh_ritz(ik, Xc[ik], resid=True)
                ev_d.append(e_)
                res_d.append(r_)
            ctx.set_f64_products(P.F64_PAIRS if pairs else P.F64_NATIVE)
            _, occ_d, e_d = P.occupations(ev_d, [1.0 / nk] * nk, w.nelectrons)
            occ_idx_d = [np.asarray(o) > 1e-8 for o in occ_d]
            accuracy = {"passes": len(hist), "seconds": acc_s, "k_points": nk,
                        "residual_target": args.acc_target,
                        "max_residual_occupied_history": hist[:5] + (["..."] if len(hist) > 10 else []) + hist[-5:],
                        "max_residual_occupied_mixed": hist[-1],
                        "max_residual_occupied_fp64": float(max(np.max(np.asarray(r)[o]) for r, o in zip(res_d, occ_idx_d))),
                        "target_met_mixed": bool(hist[-1] < args.acc_target),
                        "compared": "the converged mixed subspace iteration against one native FP64 pass from it",
                        "reference": "the FP64 GPU path",
                        "residual": "||H u - eps M u||_{M^-1} / ||u||_M of the occupied Ritz pairs",
                        "d_band_energy_per_atom_Ha": float(abs(e_m - e_d) / w.natoms),
                        "max_abs_d_eig_occupied_Ha": float(max(np.max(np.abs(np.asarray(a)[o] - np.asarray(b)[o]))
                                                               for a, b, o in zip(ev_m, ev_d, occ_idx))),
                        "occupied_states": int(sum(int(np.sum(o)) for o in occ_idx))}

    # the dominant kernel of the step (most device time per step) carries "roofline", the other
    # cell product "roofline_secondary"
    roofline, roof2 = roof_low, None
    if fp64_ms_launch is not None:
        f64_flops = ctx.product_flops(0, vslice)   # FP64-class operations of one launch (<= 64 vectors)
        f64_ach = f64_flops / (fp64_ms_launch * 1e-3) / 1e12
        fp64["product"] = {"kernel": "k_cell_apply_sf<double> + %s" % ("k_cell_apply_z3" if cplx else "k_cell_apply<double>"),
                           "ms_per_launch": fp64_ms_launch,
                           "achieved_tflops": f64_ach, "frac_of_fp64_peak": f64_ach / FP64_PEAK_DERIVED}
        mix_ach = f64_flops / (mix_ms_launch * 1e-3) / 1e12
        n_dense = nucleus_cells(w)
        n_sf = len(naug) - n_dense
        traffic = None
        if pairs and TRAFFIC_PAIR and not cplx:
            traffic = {"bytes": TRAFFIC_PAIR["sf_bytes_per_cell"] * n_sf, "source": TRAFFIC_PAIR["source"]}
        elif not pairs and TRAFFIC_FP64:
            traffic = {"bytes": TRAFFIC_FP64["bytes_per_cell"] * len(naug),
                       "source": TRAFFIC_FP64["source"] + " (scaled by cells)"}
        if pairs:
            # the refined cells (dense FP64) take a few percent of the launch; the peak is that of
            # the pair arithmetic on the FP32 pipe
            kname = ("k_cell_apply_sf<f2> + %s (FP64-class cell products: sum factorization in "
                     "FP32-pair arithmetic on single-leaf cells, FP64 dense on the refined cells)"
                     % ("k_cell_apply_z3" if cplx else "k_cell_apply<double>"))
            peak, psrc = PAIR_PEAK_DERIVED, "derived: 152 SM x 128 FP32 lanes x 2070 MHz / 12 per pair FMA x 2 flops"
        else:
            kname = ("k_cell_apply_sf + %s (FP64 cell products: sum factorization on single-leaf cells, "
                     "dense on the refined cells)" % ("k_cell_apply_z3" if cplx else "k_cell_apply<double>"))
            peak, psrc = FP64_PEAK_DERIVED, "derived: 152 SM x 2 DFMA/clk x 2 flops x 2070 MHz"
        roof_fp64 = {"kernel": kname,
                     "bound": "alu", "achieved": mix_ach, "peak": peak, "unit": "TFLOP/s",
                     "frac": mix_ach / peak,
                     "traffic": traffic["bytes"] if traffic else None,
                     "traffic_source": traffic["source"] if traffic else None,
                     "algorithmic_flops_per_launch": f64_flops, "ms_per_launch": mix_ms_launch,
                     "launches_per_step": 2 * sum(-(-v // 64) for v in nvs),
                     "peak_source": psrc,
                     "dense_equivalent_tflops": kernel_flops_per_launch(naug, vslice, cplx) / (mix_ms_launch * 1e-3) / 1e12}
        low_ms_step = per_launch_ms * klaunch / max(args.steps, 1)
        if roof_fp64["launches_per_step"] * mix_ms_launch > low_ms_step:
            roofline, roof2 = roof_fp64, roof_low
        else:
            roof2 = roof_fp64

    # end to end through the public API with host buffers (H2D of V and X0, D2H of rho and eigenvalues)
    e2e = None
    if not args.skip_e2e:
        Vh = V.cpu().pin_memory()
        X0h = [x.cpu().pin_memory() for x in X0]
        rho_h = torch.empty(rho.shape, dtype=rho.dtype).pin_memory()
        torch.cuda.synchronize()
        t_start = time.perf_counter()
        ee0 = torch.cuda.Event(enable_timing=True)
        ee1 = torch.cuda.Event(enable_timing=True)
        ee0.record(stream)
        for _ in range(args.e2e_steps):
            V.copy_(Vh, non_blocking=True)
            for ik in range(nk):
                X0[ik].copy_(X0h[ik], non_blocking=True)
            eigs_e, _ = step()
            rho_h.copy_(rho, non_blocking=True)
        ee1.record(stream)
        torch.cuda.synchronize()
        wall = (time.perf_counter() - t_start) / args.e2e_steps
        e2e_ms = ee0.elapsed_time(ee1) / args.e2e_steps
        bi = V.numel() * 8 + sum(x.numel() * x.element_size() for x in X0)
        bo = rho.numel() * 8 + sum(len(e) * 8 for e in eigs_e)
        e2e_ms = max_over_ranks(max(e2e_ms, wall * 1e3), world, "cuda")
        e2e = {"value": whole_job_tflops(flops_step, world, e2e_ms), "unit": "TFLOP/s",
               "h2d_bytes_per_step": int(bi), "d2h_bytes_per_step": int(bo), "ms_per_step": e2e_ms}

    cpu = None
    if rank == 0 and not args.skip_cpu_baseline:
        cpu = run_oracle_sample(w, args.sample_cells, steps=1, warmup=0)

    out = {"metric": "Cheb-filter TFLOP/s (dense count) & s/filter pass, mixed vs FP64 on GB300",
           "value": value, "unit": "TFLOP/s", "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
           "ms_per_step": step_ms, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
           "dtype": "c64+c128" if cplx else "f32+f64", "data": "synthetic",
           "config": {"workload": workload_text(w),
                      "arithmetic": (("mixed filter in defect form from the previous Ritz pairs (R = AQ - Q theta "
                                     "FP64-class, %d degrees of the defect on the tensor cores, Q p_m(theta) + D_m in "
                                     "FP64), FP64-class Cholesky-QR / Rayleigh-Ritz / density" % w.degree) if defect else
                                     "mixed filter (%d FP32-class degrees + last FP64-class), FP64-class Cholesky-QR / "
                                     "Rayleigh-Ritz / density" % (w.degree - 1)),
                      "start": ("Ritz pairs after %d untimed passes from random vectors" % args.init_passes
                                if defect else "random vectors"),
                      "f64_products": ("FP32 pairs on single-leaf cells (last degree and Rayleigh-Ritz H X)" if pairs
                                       else "FP64"),
                      "n_dof_per_k": int(n), "cells": int(len(naug)), "mean_n_aug": float(np.mean(naug)),
                      "l2": "inputs larger than L2 (cell matrices %.1f GB per k)" % (np.sum(naug ** 2) * 8 / 1e9),
                      "parallelism": "replicas" if world > 1 else "single GPU"},
           "filter_s_per_pass": s_per_pass, "filter_tflops": filt_tflops, "fp64": fp64, "phase_ms": phase_ms,
           "filter_launch": "batched multi-k, CUDA graph" if batched else "per k-point",
           "autotune_ms_per_degree": tune_ms,
           "filter_precision": (("BF16x%d tensor cores (FP32 defect vectors), FP64-class residual and sum" % nprod)
                                if defect else ("BF16x%d tensor cores (FP32 vectors) + last degree FP64" % nprod)
                                if args.tensor else "FP32 + last degree FP64"),
           "roofline": roofline, "roofline_secondary": roof2, "accuracy": accuracy,
           "cpu_baseline": cpu, "e2e": e2e, "clocks": clocks,
           "gpu_launches": int(launches),
           "peaks_source": src, "setup_s": setup_s}
    return out


# ----------------------------------------------------------------------------- oracle (CPU) arm
def run_oracle_sample(w, ncells_side, steps=1, warmup=0):
    """The oracle, as it stands, on a bounded sample of the same workload: a
    ncells_side^3 block of cells of the mesh at k-point 0 (cell matrices of the
    block with exact orthogonalizing coefficients), one step = build of the
    block's cell matrices + the degree-m filter pass + Cholesky-QR +
    Rayleigh-Ritz on the rows the block touches."""
    from oracle import solver
    from oracle.enrichment import Enrichment
    from oracle.mesh import Mesh
    from oracle.operators import Problem
    from oracle.quadrature import Quadrature

    xb = W.mesh_breakpoints(w)
    mesh = Mesh(w.a, xb, w.p)
    nqc, nqe, depth = w.quad_params()
    s = ncells_side
    cells = [ix + w.ncell * (iy + w.ncell * iz) for iz in range(s) for iy in range(s) for ix in range(s)]
    # the point sets of the block and of the cells around it (the orthogonalizing coefficients of the
    # block's nodes take their neighbourhood); the rest of the mesh is not tabulated
    near = sorted({f for e in cells for f in mesh.neighbours(e)})
    quad = Quadrature(mesh, w.pos, w.rc, nqc, nqe, depth, cells=near)
    R, dR = W.radial_tables(w.Z, rc=w.rc, ngrid=w.ngrid)
    enr = Enrichment(w.a, w.pos, W.orbital_lm_codes(), R, dR, w.r0, w.rc)
    k, _ = W.monkhorst_pack(w.a, w.kgrid)
    pr = Problem(mesh, quad, enr, k[0], cells=cells)
    V = np.zeros(quad.nq)   # the potential is needed only at the block's points
    for e in cells:
        sl = slice(quad.offset[e], quad.offset[e + 1])
        V[sl] = W.veff(quad.points[sl], w.a, w.pos, w.Z, w.sigma)
    # at most 64 vectors: a block of a few cells has few states below the filter's window, and more
    # filtered vectors than that are numerically dependent
    nv = min(w.nv[0], 64)
    X0 = W.random_vectors(pr.n, nv, complex_=pr.complex, seed=w.seed)
    naug = np.array([len(pr.index(e)) for e in cells])
    flops = dense_filter_flops(naug, [nv], w.degree, pr.complex)
    times = []
    for it in range(warmup + steps):
        t0 = time.perf_counter()
        pr.build(V)
        b = solver.lanczos_upper_bound(pr.apply_H, pr.apply_M, pr.apply_Minv, X0[:, 0], 10)
        Y = solver.chebyshev_filter(pr.apply_A, X0, w.degree, 0.0, b, -0.5 * max(w.Z) ** 2 - 1.0)
        Q = solver.cholqr(Y, pr.apply_M)
        solver.rayleigh_ritz(Q, pr.apply_H, pr.apply_M)
        if it >= warmup:
            times.append(time.perf_counter() - t0)
    t = float(np.mean(times))
    return {"value": flops / t / 1e12, "unit": "TFLOP/s", "cores": os.cpu_count(), "kind": "oracle",
            "s_per_step": t,
            "sample": "%d^3-cell block (%d of %d cells, %d rows, %d vectors) at k-point 0: build of the block's "
                      "cell matrices, Lanczos bound, degree-%d filter, Cholesky-QR, Rayleigh-Ritz; dense-count flops "
                      "of the block's filter / step time" % (s, len(cells), w.ncell ** 3, pr.n, nv, w.degree)}


def run_reference(args, rank, world):
    if rank != 0:
        return None
    w = W.CONFIGS[args.config]()
    res = run_oracle_sample(w, args.sample_cells, steps=args.steps, warmup=args.warmup)
    return {"impl": "reference", "metric": "Cheb-filter TFLOP/s (dense count) & s/filter pass, mixed vs FP64 on GB300",
            "value": res["value"], "unit": "TFLOP/s", "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": res["s_per_step"] * 1e3, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "c128" if is_complex(w) else "f64", "data": "synthetic",
            "config": {"workload": workload_text(w),
                       "arithmetic": "FP64 (the oracle), on a bounded sample of the workload (cpu_baseline.sample)"},
            "cpu_baseline": res,
            "e2e": {"value": res["value"], "unit": "TFLOP/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--config", default="c5", choices=["c2", "c3", "c3small", "c3mid", "c4mid", "c5", "c5mid"],
                    help="workload: c5 the large supercell the metric is quoted on (default), c3 the 8-atom cell "
                         "with 4 k-points")
    ap.add_argument("--compact", default="auto", choices=["auto", "on", "off"],
                    help="compact layout of the FP64-class cell matrices (auto: when the full copies would take "
                         "more than a quarter of the device)")
    ap.add_argument("--filter-only", action="store_true",
                    help="profiling aid: set up, then run --steps low-precision filter passes on k-point 0 only")
    ap.add_argument("--sample-cells", type=int, default=2)
    ap.add_argument("--e2e-steps", type=int, default=2)
    ap.add_argument("--skip-fp64", action="store_true")
    ap.add_argument("--per-k-filter", action="store_true", help="filter each k-point separately")
    ap.add_argument("--with-fp64", action="store_true",
                    help="with --filter-only: store the FP64 matrices too and apply H once in FP64")
    ap.add_argument("--acc-passes", type=int, default=150,
                    help="largest number of mixed subspace-iteration passes (all k) of the accuracy run")
    ap.add_argument("--acc-seconds", type=float, default=120.0,
                    help="time budget of the accuracy run (it stops at the target, the pass limit or this)")
    ap.add_argument("--acc-target", type=float, default=1e-7,
                    help="residual of the occupied states the accuracy run converges to")
    ap.add_argument("--init-passes", type=int, default=4,
                    help="untimed passes from the random start vectors to the Ritz pairs a step starts from")
    ap.add_argument("--plain-filter", action="store_true",
                    help="the plain mixed filter from the random start vectors (last degree FP64) instead of "
                         "the defect form from Ritz pairs")
    ap.add_argument("--f64-products", default="pairs", choices=["pairs", "native"],
                    help="arithmetic of the FP64-class cell products of the mixed step")
    ap.add_argument("--product-shape", type=int, default=-1, choices=[-1, 0, 1, 2],
                    help="launch shape of the FP32-pair cell products (-1: timed at first use)")
    ap.add_argument("--split", default="bf16x3", choices=["bf16x3", "bf16x6"],
                    help="bf16 split of the cell matrices for the tensor-core degrees: two parts (BF16x3, three "
                         "products) or three parts (BF16x6, six products)")
    ap.add_argument("--fp32-simt", dest="tensor", action="store_false",
                    help="FP32 SIMT cell products instead of the BF16x3 tensor-core path")
    ap.add_argument("--batched-filter", action="store_true",
                    help="with --filter-only: the batched tensor-core filter on one group of at most 128 vectors "
                         "of k-point 0 in the launch shape --filter-shape (profiling aid)")
    ap.add_argument("--filter-shape", type=int, default=-1, choices=[-1, 0, 1, 2, 3, 4, 5],
                    help="launch shape of the batched filter (oefe_set_filter_shape); -1: the default")
    ap.add_argument("--with-density", action="store_true",
                    help="with --filter-only: one density evaluation (profiling aid)")
    ap.add_argument("--with-ortho", action="store_true",
                    help="with --filter-only: two orthonormalizations of the FP64 vectors (profiling aid)")
    ap.add_argument("--skip-e2e", action="store_true")
    ap.add_argument("--skip-cpu-baseline", action="store_true")
    args = ap.parse_args()
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    if args.impl == "reference":
        out = run_reference(args, rank, world)
        if out is not None:
            print(json.dumps(out))
        return
    if world > 1:
        import torch
        torch.distributed.init_process_group("nccl")
    out = run_ours(args, rank, world)
    if rank == 0:
        print(json.dumps(out))
    if world > 1:
        import torch
        torch.distributed.destroy_process_group()


if __name__ == "__main__":
    main()
