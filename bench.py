"""Benchmark of the meshless RBF-FD leapfrog step on one GB300 (or N replicas).

Workload (default, "pulse2d-staggered-1M"): 2D TMz Gaussian-modulated pulse
on a periodic 1000 h x 1000 h square, staggered layout: 1,000,000 jittered E
nodes and 1,000,000 jittered H nodes (offset by (h/2, h/2)); curl stencils of
the 30 nearest nodes of the other set with PHS r^5 + degree-4 monomials;
hyperviscosity Delta^3 on the 57 nearest own-set nodes (PHS r^7, degree 6);
12 points per wavelength; Courant number 0.5. FP32 fields and weights
(compensated stencil sums), weights solved in FP64 on the GPU. A bench step is
one leapfrog step (H half step, E half step, source/probe/step-counter update)
over all 2M nodes; inputs (1.7 GB per step) are larger than L2.

metric: node-field updates/s = (N_E * 1 + N_H * 2) * steps / time.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import math
import os
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import workloads as W  # noqa: E402

METRIC = "node-field updates/s & HBM roofline frac, FP32 vs FP64 at stated L2 err"
UNIT = "node-field updates/s"


def _args():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5000)
    ap.add_argument("--warmup", type=int, default=20)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--nx", type=int, default=1000, help="nodes per side of each set")
    ap.add_argument("--precision", default="fp32", choices=["fp32", "fp64"])
    ap.add_argument("--plain", action="store_true", help="FP32 without compensated sums")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--accuracy-steps", type=int, default=5000,
                    help="FP32-vs-FP64 (GPU) relative L2 error after this many steps (0: skip)")
    ap.add_argument("--no-fp64", action="store_true", help="skip the FP64 step and the accuracy runs")
    ap.add_argument("--cube-steps", type=int, default=2000,
                    help="steps of the 3D 200^3 PEC-cube workload (0: skip)")
    ap.add_argument("--cube-nx", type=int, default=200, help="nodes per side of the 3D cube")
    ap.add_argument("--yee-grid", type=int, default=8192, help="cells per side of the FDTD roofline grid")
    ap.add_argument("--batched-ndom", type=int, default=256, help="domains of the batched workload")
    ap.add_argument("--no-extra", action="store_true", help="skip the cavity (FP64) and adjoint sections")
    ap.add_argument("--only", default="all", choices=["all", "batched", "cube3d", "cavity", "adjoint", "dispersion", "hv_search", "yee"],
                    help="run one section alone (profiling); prints that section as the JSON line")
    ap.add_argument("--adjoint-steps", type=int, default=4000,
                    help="steps of the differentiation workload (--only adjoint)")
    ap.add_argument("--batched-steps", type=int, default=3000,
                    help="steps of the batched 256-domain x 16-RHS workload (0: skip)")
    ap.add_argument("--l2-keep", type=float, default=None,
                    help="fraction of the stencil streams kept in L2 for the headline and adjoint "
                         "simulations (mfd_sim_set_l2_keep; default: sized from the L2)")
    return ap.parse_args()


def config(name):
    """One workload's parameters (configs/<name>.json)."""
    return json.load(open(os.path.join(ROOT, "configs", name + ".json")))


C1, C2, C3, C4, C5 = (config(x) for x in ("c1_cavity", "c2_pulse", "c3_cube", "c4_batched", "c5_adjoint"))
CAV_L = float(C1["nodes"]["shape"][0] - 1)  # side of the cavity: the PEC box's wall nodes sit at 0 and L
PARAMS = dict(S=C2["courant"], n=C2["curl"]["n"], k=C2["curl"]["phs_k"], m=C2["curl"]["poly_m"],
              alpha=C2["hv"]["alpha"], c=C2["hv"]["c"], wavelength=C2["wavelength"])


def pulse_fields(e, h, nx, dt):
    S = PARAMS["S"]
    _, _, _, c0, eta0 = W.units(S)
    lam = PARAMS["wavelength"]
    ez, _, _ = W.gaussian_pulse(e.xyz, nx, nx / 2, 2 * lam, c0, eta0, dt, lam)
    _, hx, hy = W.gaussian_pulse(h.xyz, nx, nx / 2, 2 * lam, c0, eta0, dt, lam)
    return ez, hx, hy


def node_sets(nx):
    nd = C2["nodes"]
    e = W.periodic_box((nx, nx), nd["jitter"], nd["e_seed"], seed_line_y=nx // 2)
    h = W.periodic_box((nx, nx), nd["jitter"], nd["h_seed"], offset=tuple(nd["h_offset"]))
    return e, h


def algorithmic_bytes(n, nhv, s):
    """Compulsory bytes per node of each half step (staggered; int32 indices, s bytes per real).
    H pass: indices 4 (n + N_h), weights s (2 n + N_h), fields Ez (gathered once) + H read + H written.
    E pass: same streams; fields H' + Ez read, Ez written."""
    h = 4 * (n + nhv) + s * (2 * n + nhv) + 5 * s
    e = 4 * (n + nhv) + s * (2 * n + nhv) + 4 * s
    return h, e


def colloc_bytes(n, nhv, s):
    """Algorithmic bytes per node of each half step of the collocated 2D step (s bytes per
    real; neighbour gathers counted once; each field read once and written once). H pass:
    the shared index row of max(n, N_h) int32 entries, curl weights 2 n s and HV weights
    N_h s, Ez, Hx, Hy read and E*, Hx', Hy' written (6 s). E pass: the first n entries of
    the row, 2 n s of curl weights, E* and ce read and Ez written with H' gathered (4 s).
    (The {Ez, Hx, Hy, ce} layout moves a whole 16-byte block per node and pass: 24 B more.)"""
    h = 4 * max(n, nhv) + s * (2 * n + nhv) + 6 * s
    e = 4 * n + s * 2 * n + 4 * s
    return h, e


def solve_flops(K, nout):
    """FP64 flops of one local weight system solved by Gaussian elimination on its
    K x (K + nout) augmented matrix (an FMA counted as two): the eliminations
    sum_p 2 (K - 1 - p)(K + nout - 1 - p), plus nout back substitutions of K^2."""
    return sum(2 * (K - 1 - p) * (K + nout - 1 - p) for p in range(K)) + nout * K * K


def poly_count(m, dim=2):
    """Monomials of total degree <= m in dim variables."""
    return math.comb(m + dim, dim)


def build_weights(M, ctx, e, h):
    """Node sets, kNN stencils and FP64 weights of the staggered workload (setup, timed apart)."""
    n, k, m, alpha = (PARAMS[x] for x in ("n", "k", "m", "alpha"))
    nhv = 2 * math.comb(2 * alpha + 2, 2) + 1
    t = time.time()
    de, dh = M.Nodes(ctx, e.xyz, e.period), M.Nodes(ctx, h.xyz, h.period)
    s_he, s_hh = M.Stencils(dh, de, n), M.Stencils(dh, dh, nhv)
    s_eh, s_ee = M.Stencils(de, dh, n), M.Stencils(de, de, nhv)
    ctx.sync()
    t_knn = time.time() - t
    t = time.time()
    hc = M.Weights(s_he, n, k, m, M.MFD_OP_GRAD)
    hv = M.Weights(s_hh, nhv, 2 * alpha + 1, 2 * alpha, M.MFD_OP_LAP_POW, alpha)
    ec = M.Weights(s_eh, n, k, m, M.MFD_OP_GRAD)
    ev = M.Weights(s_ee, nhv, 2 * alpha + 1, 2 * alpha, M.MFD_OP_LAP_POW, alpha)
    ctx.sync()
    t_w = time.time() - t
    return (hc, hv, ec, ev), dict(morton_knn_s=round(t_knn, 3), weights_fp64_s=round(t_w, 3)), nhv


def make_sim(M, ctx, wts, precision, compensated):
    S, c, alpha = PARAMS["S"], PARAMS["c"], PARAMS["alpha"]
    dt, eps0, mu0, c0, eta0 = W.units(S)
    gamma = c * (-1) ** (alpha - 1)
    hc, hv, ec, ev = wts
    return M.Sim(ctx, 2, precision, dt, eps0, mu0, gamma, hc, hv, ec, ev, compensated=compensated)


class ClockSampler:
    """Samples nvidia-smi clocks and throttle reasons while the timed region runs."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "100"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except Exception:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if not self.proc:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"], "samples": 0}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        sm, smax, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            p = [x.strip() for x in ln.split(",")]
            if len(p) < 9:
                continue
            try:
                sm.append(float(p[1]))
                smax = float(p[2])
            except ValueError:
                continue
            for nm, v in zip(names, p[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        return {"sm_mhz": float(np.median(sm)) if sm else None, "sm_max_mhz": smax,
                "reasons": sorted(reasons), "samples": len(sm)}


def aggregate(elapsed_s, units, dist=None):
    """Whole-job throughput of N replicas: the slowest rank's time (max over
    ranks, all-reduced) and value = units x world / that time. Returns
    (max elapsed seconds, value)."""
    world = 1
    if dist is not None and dist.is_initialized():
        import torch
        world = dist.get_world_size()
        dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
        t = torch.tensor([float(elapsed_s)], dtype=torch.float64, device=dev)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        elapsed_s = float(t.item())
    return elapsed_s, units * world / elapsed_s


def _sm_max_mhz():
    """The maximum SM clock (MHz) from the measured peaks, else the GB300's 2070 MHz."""
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return float(json.load(f).get("sm_max_mhz", 2070.0))
    except (OSError, ValueError):
        return 2070.0


def peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        d = json.load(open(p))
        return d.get("hbm_gbs", 6800.0), "measured"
    return 6800.0, "fallback"


def traffic_record(kernel, s, algorithmic):
    """DRAM bytes per launch of `kernel` (s-byte reals): the ratio of DRAM bytes
    to algorithmic bytes that ncu measured on a smaller case of the same
    kernel (profiles/traffic.json) times this launch's algorithmic bytes, if
    the source files that define the kernel are unchanged since that capture
    (else None)."""
    p = os.path.join(ROOT, "profiles", "traffic.json")
    if not os.path.exists(p):
        return None
    rec = json.load(open(p)).get("kernels", {}).get(f"{kernel}_fp{8 * s}")
    if not rec or rec.get("sha") != sources_sha(rec.get("sources", [])):
        return None
    return round(rec["ratio"] * algorithmic) if "ratio" in rec else rec.get("bytes")


def sources_sha(files):
    hsh = hashlib.sha256()
    cs = os.path.join(ROOT, "paper_2508_18205_gb300", "csrc")
    for f in sorted(files):
        hsh.update(open(os.path.join(cs, f), "rb").read())
    return hsh.hexdigest()[:16]


def cpu_baseline(budget_s=20.0):
    """The oracle (FP64, OpenMP on the host cores) on a bounded sample of the
    same workload: a 160 x 160 periodic staggered sub-square with the same
    stencils, stepped for about budget_s seconds."""
    import oracle as O
    S, n, k, m, alpha, c = (PARAMS[x] for x in ("S", "n", "k", "m", "alpha", "c"))
    dt, eps0, mu0, c0, eta0 = W.units(S)
    nx = 160
    e, h = node_sets(nx)
    prob = O.tmz_staggered(e, h, n, k, m, alpha, dt, eps0, mu0, c * (-1) ** (alpha - 1))
    ez, hx, hy = pulse_fields(e, h, nx, dt)
    t = time.time()
    O.run_tmz(prob, ez, hx, hy, 5)
    per = (time.time() - t) / 5
    steps = max(5, int(budget_s / max(per, 1e-6)))
    t = time.time()
    O.run_tmz(prob, ez, hx, hy, steps)
    el = time.time() - t
    updates = (e.n + 2 * h.n) * steps
    return {"value": updates / el, "unit": UNIT, "cores": O.threads(), "kind": "oracle",
            "sample": f"{nx}x{nx}+{nx}x{nx} staggered periodic sub-square, same stencils, {steps} steps "
                      f"in {el:.1f} s (FP64)",
            "cavity_fp64": cavity_cpu(O)}


def _rel(a, b):
    return float(np.linalg.norm(np.asarray(a) - np.asarray(b)) / np.linalg.norm(b))


def _maxabs(a, b):
    return float(np.max(np.abs(np.asarray(a) - np.asarray(b))))


def oracle_checks(gpu):
    """Relative L2 and largest absolute error of every workload's GPU results
    against the FP64 oracle, which runs here on the host cores from the same
    seeded inputs (node sets, fields, sources, materials) the GPU sections
    used; nothing the GPU computed is an input of the oracle. gpu: the
    host-side results the GPU sections kept (their "_gpu" entries)."""
    import oracle as O
    out = {}
    t_all = time.perf_counter()
    # headline problem on a 160^2 + 160^2 sub-square, the whole 5000 steps
    g = gpu.get("pulse_reduced")
    if g:
        t = time.perf_counter()
        S, n, k, m, alpha, c = (PARAMS[x] for x in ("S", "n", "k", "m", "alpha", "c"))
        dt, eps0, mu0, c0, eta0 = W.units(S)
        e, h = node_sets(g["nx"])
        prob = O.tmz_staggered(e, h, n, k, m, alpha, dt, eps0, mu0, c * (-1) ** (alpha - 1))
        ez, hx, hy = pulse_fields(e, h, g["nx"], dt)
        probes = W.interior_nodes(e, 16, 24)
        ref, rp, every = [ez, hx, hy], [], g["every"]
        snaps = []
        for kk in range(g["steps"] // every):
            o = O.run_tmz(prob, *ref, every, step0=kk * every, probes=probes)
            ref = list(o[:3])
            rp.append(o[3])
            snaps.append(np.concatenate(ref))
        rp = np.concatenate(rp)
        res = {"workload": f"pulse2d-staggered-{g['nx']}x{g['nx']}x2 (same stencils and pulse as the headline)",
               "steps": g["steps"], "compared_every": every}
        for tag in ("fp32_compensated", "fp32_plain", "fp64"):
            errs = [_rel(a, b) for a, b in zip(g[tag]["snaps"], snaps)]
            res[tag] = {"rel_l2_max_over_checks": max(errs), "rel_l2_end": errs[-1],
                        "max_abs_end": _maxabs(g[tag]["snaps"][-1], snaps[-1]),
                        "probe_rel_l2": _rel(g[tag]["probes"], rp)}
        res["oracle_s"] = round(time.perf_counter() - t, 2)
        out["pulse2d_staggered"] = res
    # the plain method's cavity (FP64), the whole workload
    g = gpu.get("cavity_fp64")
    if g:
        S, c, nodes, (n, k, m, alpha) = cavity_setup()
        dt, eps0, mu0, c0, eta0 = W.units(S)
        prob, _ = O.tmz_collocated(nodes, n, k, m, alpha, dt, eps0, mu0, -c)
        ez, hx, hy = W.tm11_fields(nodes.xyz, CAV_L, c0, mu0, 0.0, -0.5 * dt)
        ez[nodes.pec == 1] = 0
        o = O.run_tmz(prob, ez, hx, hy, g["steps"], probes=W.interior_nodes(nodes, C1["probes"]["count"], C1["probes"]["seed"]))
        ref = np.concatenate(o[:3])
        out["cavity_fp64"] = {"workload": "cavity TM11, 100x100 PEC, n=12, FP64 (whole workload)",
                              "steps": g["steps"], "rel_l2": _rel(g["fields"], ref),
                              "max_abs": _maxabs(g["fields"], ref), "probe_rel_l2": _rel(g["probes"], o[3])}
    # 3D PEC cube: the first step at full size (sampled nodes far from the walls,
    # and sampled nodes in a corner, where the stencils take images) and a whole
    # run of a 32^3 cube
    g = gpu.get("cube3d")
    if g:
        t = time.perf_counter()
        S, cc, n, k, m, alpha = (CUBE[x] for x in ("S", "c", "n", "k", "m", "alpha"))
        dt, eps0, mu0, c0, eta0 = W.units(S)
        sm = g["sampled"]
        nodes = sm["nodes"]
        ids = sm["ids_in"]
        # away from the walls no stencil of a node the step reads takes an image:
        # the plain stencils of the box's own nodes
        RE, RH, hs = O.max3d_sample_step(nodes, ids, n, k, m, alpha, dt, eps0, mu0, -cc, sm["E0"], sm["H0"],
                                         eps_r=sm["eps_r"], h_ids=ids)
        RHi = RH[:, np.searchsorted(hs, ids)]
        got = np.concatenate([sm["E1_in"].ravel(), sm["H1_in"].ravel()])
        ref = np.concatenate([RE.ravel(), RHi.ravel()])
        res = {"workload": "cube3d-pec (walls by images)", "full_size_first_step_interior": {
            "nodes": nodes.n, "sampled_nodes": len(ids), "rel_l2": _rel(got, ref), "max_abs": _maxabs(got, ref)}}
        # the corner: the oracle's image scheme on the 20^3 cells at the corner,
        # a PEC box of its own whose far walls lie beyond what the sampled
        # nodes' first step reads (two stencil radii, under 6 spacings)
        cell = np.floor(nodes.xyz).astype(np.int64)
        sub = np.nonzero(np.all(cell < 20, axis=1))[0]
        crop = W.NodeSet(xyz=nodes.xyz[sub], pec=np.zeros(len(sub), np.uint8), period=np.zeros(3),
                         box_lo=np.zeros(3), box_hi=np.full(3, 20.0), normal_axes=np.zeros(len(sub), np.uint8))
        prob = O.max3d_images(crop, n, k, m, alpha, dt, eps0, mu0, -cc, eps_r=sm["eps_r"][sub], n_wall=CUBE["n_wall"])
        RE, RH, _, _ = O.run_3d(prob, sm["E0"][:, sub], sm["H0"][:, sub], 1)
        at = np.searchsorted(sub, sm["ids_wall"])
        got = np.concatenate([sm["E1_wall"].ravel(), sm["H1_wall"].ravel()])
        ref = np.concatenate([RE[:, at].ravel(), RH[:, at].ravel()])
        res["full_size_first_step_corner"] = {"sampled_nodes": len(at), "rel_l2": _rel(got, ref),
                                              "max_abs": _maxabs(got, ref)}
        sg = g["small"]
        RE, RH, en = O.run_3d_images(sg["nodes"], n, k, m, alpha, dt, eps0, mu0, -cc, sg["E0"], sg["H0"],
                                     sg["steps"], eps_r=sg["eps_r"], energy=True, n_wall=CUBE["n_wall"])
        ref = np.concatenate([RE, RH])
        u = en / en[0]
        res[f"cube_{sg['nx']}^3_whole_run"] = {"steps": sg["steps"], "rel_l2": _rel(sg["fields"], ref),
                                              "max_abs": _maxabs(sg["fields"], ref),
                                              "oracle_energy_rel": {"min": float(u.min()), "max": float(u.max()),
                                                                    "end": float(u[-1])}}
        res["oracle_s"] = round(time.perf_counter() - t, 2)
        out["cube3d"] = res
    # batched: whole domains (one of each stencil size), four right-hand sides each
    g = gpu.get("batched")
    if g:
        t = time.perf_counter()
        S = C4["courant"]
        dt, eps0, mu0, c0, eta0 = W.units(S)
        doms = []
        worst = 0.0
        for D in g["domains"]:
            ns, n = D["nodes"], D["n"]
            prob, _ = O.tmz_collocated(ns, n, C4["curl"]["phs_k"], W.poly_degree_for(n), C4["hv"]["alpha"], dt, eps0,
                                       mu0, -g["c"], nh_override=C4["hv"]["n"])
            z = np.zeros(ns.n)
            got, ref = [], []
            for j, r in enumerate(D["rhs"]):
                sel = D["src"].rhs == r
                src = D["src"]
                sub = W.Sources(node=src.node[sel], rhs=src.rhs[sel], amp=src.amp[sel], f0=src.f0[sel],
                                t0=src.t0[sel])
                o = O.run_tmz(prob, z, z, z, g["steps"], sources=sub)
                ref.append(np.concatenate(o[:3]))
                got.append(np.concatenate([D["ez"][:, j], D["hx"][:, j], D["hy"][:, j]]))
            got, ref = np.concatenate(got), np.concatenate(ref)
            e_ = _rel(got, ref)
            worst = max(worst, e_)
            doms.append({"domain": D["dom"], "nodes": ns.n, "n": n, "rhs": D["rhs"], "rel_l2": e_,
                         "max_abs": _maxabs(got, ref)})
        out["batched"] = {"steps": g["steps"], "domains": doms, "rel_l2_max": worst,
                          "oracle_s": round(time.perf_counter() - t, 2)}
    # adjoint: the gradient of the FP32 GPU adjoint against the FP64 oracle adjoint
    g = gpu.get("adjoint")
    if g:
        P = _adjoint_problem(g["nx"])
        dt, eps0, mu0, c0, eta0 = W.units(P["S"])
        n, k, m, nh, alpha = P["stencil"]
        prob, _ = O.tmz_collocated(P["nodes"], n, k, m, alpha, dt, eps0, mu0, -P["c"], eps_r=P["eps"],
                                   nh_override=nh)
        z = np.zeros(P["nodes"].n)
        J, ge, ga = O.grad_tmz(prob, z, z, z, g["steps"], P["src"], P["probes"])
        out["adjoint"] = {"workload": f"adjoint {g['nx']}x{g['nx']} PEC, n=20, FP32 GPU vs FP64 oracle",
                          "steps": g["steps"], "J_rel": abs(g["J"] - J) / abs(J), "g_eps_rel_l2": _rel(g["g_eps"], ge),
                          "g_eps_max_abs": _maxabs(g["g_eps"], ge), "g_amp_rel_l2": _rel(g["g_amp"], ga)}
    out["oracle_s_total"] = round(time.perf_counter() - t_all, 2)
    out["cores"] = O.threads()
    return out


def cavity_cpu(O, steps=1000):
    """The oracle on the whole FP64 cavity workload of cavity() (100 x 100 PEC
    square, n = 12, Delta^2 HV, TM11 mode, 1000 steps), on all host cores and
    on one thread, with its relative L2 error against the exact mode."""
    S, c, nodes, (n, k, m, alpha) = cavity_setup()
    dt, eps0, mu0, c0, eta0 = W.units(S)
    prob, _ = O.tmz_collocated(nodes, n, k, m, alpha, dt, eps0, mu0, -c)
    ez, hx, hy = W.tm11_fields(nodes.xyz, CAV_L, c0, mu0, 0.0, -0.5 * dt)
    ez[nodes.pec == 1] = 0
    cores = O.threads()
    out = {"workload": "cavity TM11, 100x100 PEC, n=12, FP64, 1000 steps"}
    try:
        for key, th in (("all_cores", cores), ("one_thread", 1)):
            O.threads(th)
            t = time.perf_counter()
            res = O.run_tmz(prob, ez, hx, hy, steps)
            el = time.perf_counter() - t
            out[key] = {"value": nodes.n * 3 * steps / el, "unit": UNIT, "cores": th,
                        "ms_per_step": el / steps * 1e3}
    finally:
        O.threads(cores)
    T = steps * dt
    ea, xa, ya = W.tm11_fields(nodes.xyz, CAV_L, c0, mu0, T, T - 0.5 * dt)
    got, ref = np.concatenate(res[:3]), np.concatenate([ea, xa, ya])
    out["rel_l2_vs_exact_mode"] = float(np.linalg.norm(got - ref) / np.linalg.norm(ref))
    return out


def run_reference(a, rank, world):
    """The reference arm: the FP64 oracle as it stands, on the host cores, one
    bench step = one leapfrog step of a bounded sample of the workload (a
    160 x 160 + 160 x 160 staggered periodic sub-square with the same stencils
    and coefficients). Rank 0 alone runs it."""
    if rank != 0:
        return
    import oracle as O
    O.build()
    S, n, k, m, alpha, c = (PARAMS[x] for x in ("S", "n", "k", "m", "alpha", "c"))
    dt, eps0, mu0, c0, eta0 = W.units(S)
    nx = 160
    e, h = node_sets(nx)
    t0 = time.time()
    prob = O.tmz_staggered(e, h, n, k, m, alpha, dt, eps0, mu0, c * (-1) ** (alpha - 1))
    setup = time.time() - t0
    ez, hx, hy = pulse_fields(e, h, nx, dt)
    if a.warmup:
        ez, hx, hy, _, _ = O.run_tmz(prob, ez, hx, hy, a.warmup)
    t0 = time.perf_counter()
    O.run_tmz(prob, ez, hx, hy, a.steps, step0=a.warmup)
    el = time.perf_counter() - t0
    v = (e.n + 2 * h.n) * a.steps / el
    cb = {"value": v, "unit": UNIT, "cores": O.threads(), "kind": "oracle",
          "sample": f"{nx}x{nx}+{nx}x{nx} staggered periodic sub-square of the workload, same stencils, "
                    f"{a.steps} FP64 steps in {el:.2f} s (setup {setup:.1f} s)"}
    line = {"metric": METRIC, "value": v, "unit": UNIT, "n_gpus": a.gpus, "steps": a.steps, "warmup": a.warmup,
            "ms_per_step": el / a.steps * 1e3, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "f64", "data": "synthetic", "impl": "reference",
            "config": {"workload": f"pulse2d-staggered-{a.nx}x{a.nx}x2 (bounded sample: {nx}x{nx}x2)",
                       "nodes_per_set": nx * nx},
            "cpu_baseline": cb,
            "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def main():
    a = _args()
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if a.impl == "reference":
        return run_reference(a, rank, world)
    import torch
    import paper_2508_18205_gb300 as M
    from paper_2508_18205_gb300 import build as B
    B.build()
    torch.cuda.set_device(local)
    if a.only != "all":
        ctx = M.Ctx(local)
        peak, peak_kind = peaks()
        if a.only == "batched":
            r = batched(M, ctx, a.batched_steps, peak, peak_kind, ndom=a.batched_ndom)
        elif a.only == "cavity":
            r = cavity(M, ctx)
        elif a.only == "adjoint":
            r = adjoint(M, ctx, steps=a.adjoint_steps, l2_keep=a.l2_keep)
        elif a.only == "hv_search":
            r = hv_search(M, ctx)
        elif a.only == "yee":
            r = yee(M, ctx, peak, peak_kind, big=a.yee_grid)
        elif a.only == "dispersion":
            e, h = node_sets(a.nx)
            wts, _, _ = build_weights(M, ctx, e, h)
            ez, hx, hy = pulse_fields(e, h, a.nx, W.units(PARAMS["S"])[0])

            def reset(s_, cap):
                for comp_, v in ((M.MFD_EZ, ez), (M.MFD_HX, hx), (M.MFD_HY, hy)):
                    s_.set_field(comp_, v)
                s_.set_probes(W.interior_nodes(e, 16, 24), cap)
            r = dispersion(M, ctx, wts, e, reset, not a.plain)
        else:
            r = cube3d(M, ctx, a.cube_steps, peak, peak_kind, nx=a.cube_nx)
        r.pop("_gpu", None)
        print(json.dumps(r), flush=True)
        return
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    prec = M.MFD_FP64 if a.precision == "fp64" else M.MFD_FP32
    comp = prec == M.MFD_FP32 and not a.plain
    nx = a.nx
    e, h = node_sets(nx)
    ctx = M.Ctx(local)
    wts, setup, nhv = build_weights(M, ctx, e, h)
    # the batched FP64 weight solve (setup) against the FP64 FMA peak measured on this GPU:
    # curl systems n + M_m (two right-hand sides) and HV systems N_h + M_{2 alpha} (one), per node
    g64_peak = M.fma_peak(local)[0]
    sys_fl = (solve_flops(PARAMS["n"] + poly_count(PARAMS["m"]), 2)
              + solve_flops(nhv + poly_count(2 * PARAMS["alpha"]), 1)) * (e.n + h.n)
    weights_roof = {"bound": "alu", "achieved": sys_fl / setup["weights_fp64_s"] / 1e12, "peak": g64_peak / 1e3,
                    "unit": "TFLOP/s", "frac": sys_fl / setup["weights_fp64_s"] / 1e9 / g64_peak,
                    "flops": sys_fl, "seconds": setup["weights_fp64_s"], "kernel": "k_weights",
                    "peak_kind": "measured live (FP64 FMA chains, mfd_fma_peak)",
                    "note": "elimination flops only (the PHS and monomial evaluations that assemble the systems are not counted)"}
    sim = make_sim(M, ctx, wts, prec, comp)
    if a.l2_keep is not None:
        sim.set_l2_keep(a.l2_keep)
    S = PARAMS["S"]
    dt = W.units(S)[0]
    ez, hx, hy = pulse_fields(e, h, nx, dt)
    probes = W.interior_nodes(e, 16, 24)

    def reset(s_, cap):
        s_.set_field(M.MFD_EZ, ez)
        s_.set_field(M.MFD_HX, hx)
        s_.set_field(M.MFD_HY, hy)
        s_.set_probes(probes, cap)

    reset(sim, a.steps + a.warmup + 8)
    u0 = sim.energy()  # Eq. 20 of the initial state
    blocks = sim.autotune(20)
    stream = ctx.torch_stream()
    sim.step(a.warmup)
    sim.step_timed(min(a.steps, 64))  # creates the per-launch event pool
    sampler = ClockSampler(local)
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    sampler.start()
    t_start = torch.cuda.Event(enable_timing=True)
    t_end = torch.cuda.Event(enable_timing=True)
    t_start.record(stream)
    sim.step(a.steps)                 # production path: graph replay
    t_end.record(stream)
    torch.cuda.synchronize()
    elapsed = t_start.elapsed_time(t_end) / 1e3
    # per-kernel durations: the same number of steps, every launch bracketed by CUDA events
    ms = sim.step_timed(a.steps)
    clocks = sampler.stop()
    u_rel = sim.energy() / u0  # after warm-up + min(K, 64) + 2K steps
    per_step_updates = e.n + 2 * h.n
    elapsed, value = aggregate(elapsed, per_step_updates * a.steps, dist)
    if dist:
        dist.barrier()
    s = 8 if prec == M.MFD_FP64 else 4
    peak, peak_kind = peaks()
    stats = sim.index_stats()
    roof = roofline(ms, a.steps, e, h, nhv, s, peak, peak_kind, stats)
    # the same steps with 32-bit indices everywhere, for comparison (bit-identical fields)
    k32 = min(a.steps, 1000)
    sim.set_index_format(M.MFD_INDEX_I32)
    sim.step(4)
    torch.cuda.synchronize()
    t_start.record(stream)
    sim.step(k32)
    t_end.record(stream)
    torch.cuda.synchronize()
    i32_ms = t_start.elapsed_time(t_end) / k32
    sim.set_index_format(M.MFD_INDEX_Q16)
    step_bytes = format_bytes(PARAMS["n"], nhv, s, stats)
    step_gb = (step_bytes[0] * h.n + step_bytes[1] * e.n) / 1e9
    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": a.steps,
            "warmup": a.warmup, "ms_per_step": elapsed / a.steps * 1e3, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64" if prec == M.MFD_FP64 else "f32",
            "data": "synthetic",
            "config": {"workload": f"pulse2d-staggered-{nx}x{nx}x2",
                       "nodes_per_set": nx * nx, "layout": "staggered", "curl_stencil": PARAMS["n"],
                       "hv_stencil": nhv, "phs": PARAMS["k"], "poly_m": PARAMS["m"], "alpha": PARAMS["alpha"],
                       "courant": S, "compensated": comp, "l2_flush": f"inputs larger than L2 ({step_gb:.2f} GB/step)",
                       "parallelism": f"replicas{world}", "setup_s": setup, "weights_roofline": weights_roof,
                       "autotuned_blocks": {"h_pass": blocks[0], "e_pass": blocks[1]},
                       "l2_keep": sim.l2_keep},
            "roofline": roof, "clocks": clocks, "gpu_launches": 3 * a.steps,
            "energy_rel_end": {"u": u_rel, "after_steps": a.warmup + min(a.steps, 64) + 2 * a.steps},
            "event_timed_ms_per_step": (ms[0] + ms[1]) / a.steps,
            "index_i32": {"ms_per_step": i32_ms, "steps": k32,
                          "value": per_step_updates / (i32_ms / 1e3) * world}}
    # the single-GPU sections (FP64 step, accuracy, the other workloads, the CPU baseline) run
    # at N = 1 only: with replicas they would hold every GPU while rank 0 alone works
    solo = world == 1
    # the plain FP64 GPU step on the same GPU, and FP32 accuracy against it
    if solo and not a.no_fp64 and prec == M.MFD_FP32:
        k64 = min(a.steps, 1000)
        s64 = make_sim(M, ctx, wts, M.MFD_FP64, False)
        reset(s64, 8)
        s64.autotune(10)
        s64.step(a.warmup)
        torch.cuda.synchronize()
        t0 = torch.cuda.Event(enable_timing=True)
        t1 = torch.cuda.Event(enable_timing=True)
        t0.record(stream)
        s64.step(k64)
        t1.record(stream)
        torch.cuda.synchronize()
        el64 = t0.elapsed_time(t1) / 1e3
        ms64 = s64.step_timed(k64)
        g64, g32 = M.fma_peak(local)
        nh_ = h.n
        # FP64 flops per launch: curl 2 n + HV 2 N_h FMAs per H node, curl 2 n + HV N_h per E node
        fl_h = 2.0 * nh_ * (2 * PARAMS["n"] + 2 * nhv)
        fl_e = 2.0 * e.n * (2 * PARAMS["n"] + nhv)
        th, te = ms64[0] / k64 / 1e3, ms64[1] / k64 / 1e3
        dom_fl, dom_t, kn = (fl_h, th, "k_h_stag") if th >= te else (fl_e, te, "k_e_stag")
        line["fp64"] = {"value": per_step_updates * k64 / el64, "unit": UNIT, "steps": k64,
                        "ms_per_step": el64 / k64 * 1e3,
                        "roofline": {"bound": "alu", "achieved": dom_fl / dom_t / 1e12, "peak": g64 / 1e3,
                                     "unit": "TFLOP/s", "frac": dom_fl / dom_t / 1e9 / g64, "traffic": None,
                                     "kernel": kn, "peak_kind": "measured live (FP64 FMA chains, mfd_fma_peak)",
                                     "flops_per_launch": dom_fl, "avg_launch_ms": dom_t * 1e3,
                                     "hbm": roofline(ms64, k64, e, h, nhv, 8, peak, peak_kind, stats)},
                        "fma_peak_gflops": {"fp64": g64, "fp32": g32}}
        del s64
        if a.accuracy_steps:
            line["accuracy"] = accuracy(M, ctx, wts, a.accuracy_steps, reset)
    gpu_kept = {}
    if solo and not a.no_fp64 and not a.no_cpu and prec == M.MFD_FP32 and a.accuracy_steps:
        gpu_kept["pulse_reduced"] = pulse_reduced_gpu(M, ctx, 160, a.accuracy_steps)
    if solo and not a.no_extra:
        line["dispersion"] = dispersion(M, ctx, wts, e, reset, comp)
    if solo and a.batched_steps:
        line["batched"] = batched(M, ctx, a.batched_steps, peak, peak_kind)
    if solo and a.cube_steps:
        line["cube3d"] = cube3d(M, ctx, a.cube_steps, peak, peak_kind)
    if solo and not a.no_extra:
        line["cavity_fp64"] = cavity(M, ctx)
        line["adjoint"] = adjoint(M, ctx, l2_keep=a.l2_keep)
        line["hv_search"] = hv_search(M, ctx)
        line["yee"] = yee(M, ctx, peak, peak_kind)
    # end to end through the public API: host fields in, steps, host Ez + probes out
    if not a.no_e2e:
        pin = [torch.empty(x.shape[0], dtype=torch.float64, pin_memory=True) for x in (ez, hx, hy)]
        for t_, x in zip(pin, (ez, hx, hy)):
            t_.numpy()[:] = x
        out = torch.empty(e.n, dtype=torch.float64, pin_memory=True)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        sim.set_field(M.MFD_EZ, pin[0].numpy())
        sim.set_field(M.MFD_HX, pin[1].numpy())
        sim.set_field(M.MFD_HY, pin[2].numpy())
        sim.set_probes(probes, a.steps)
        sim.step(a.steps)
        sim.ctx.sync()
        res = sim.read_probes()
        lib = M.lib()
        import ctypes
        M._ck(lib.mfd_get_field(sim.h, M.MFD_EZ, 0, ctypes.c_void_p(out.data_ptr())))
        el = time.perf_counter() - t0
        h2d = 8 * (e.n + 2 * h.n)
        d2h = 8 * e.n + res.nbytes
        line["e2e"] = {"value": per_step_updates * a.steps / el * world, "unit": UNIT,
                       "h2d_bytes_per_step": h2d / a.steps, "d2h_bytes_per_step": d2h / a.steps,
                       "wall_s": el}
    for key in ("cavity_fp64", "cube3d", "batched", "adjoint"):
        if isinstance(line.get(key), dict) and "_gpu" in line[key]:
            gpu_kept[key] = line[key].pop("_gpu")
    if solo and not a.no_cpu:
        try:
            line["cpu_baseline"] = cpu_baseline()
        except Exception as ex:  # the oracle is test infrastructure; report why it is missing
            line["cpu_baseline"] = {"value": None, "error": str(ex)}
        try:
            line["accuracy_vs_oracle"] = oracle_checks(gpu_kept)
        except Exception as ex:
            line["accuracy_vs_oracle"] = {"error": str(ex)}
    del gpu_kept
    if rank == 0:
        print(json.dumps(line), flush=True)
    if dist:
        dist.destroy_process_group()


def format_bytes(n, nhv, s, stats):
    """Compulsory bytes per node of each half step in the 16-bit index format
    (mfd_sim_set_index_format): 2 bytes per entry, 4 in the slices that keep
    32-bit entries, plus the two 4-byte bases per slice and stream."""
    out = []
    for p, fields in (("h", 5), ("e", 4)):
        sl, wc, wv = stats[p]
        if sl == 0:  # no 16-bit streams: 32-bit entries
            out.append(algorithmic_bytes(n, nhv, s)[0 if p == "h" else 1])
            continue
        idx = sum((2 + 2 * w / sl) * k for w, k in ((wc, n), (wv, nhv))) + 2 * 8 / 32
        out.append(idx + s * (2 * n + nhv) + fields * s)
    return tuple(out)


def roofline(ms, steps, e, h, nhv, s, peak, peak_kind, stats=None):
    """Dominant half-step kernel: compulsory bytes per launch / its average
    event-timed duration. The compulsory bytes are those of the index format
    the kernels read: with 16-bit index streams (index statistics given and
    nonzero) 2 bytes per entry (4 in slices that keep 32-bit entries) plus the
    slice bases, else 32-bit indices. The count with 32-bit indices everywhere
    (the per-node figure of the method's layout, 836 / 832 B at n = 30,
    N_h = 57 in FP32) is reported beside it."""
    bh, be = algorithmic_bytes(PARAMS["n"], nhv, s)
    h_avg = ms[0] / steps / 1e3
    e_avg = ms[1] / steps / 1e3
    dom = "h" if h_avg >= e_avg else "e"
    dom_t = max(h_avg, e_avg)
    other_t = min(h_avg, e_avg)
    i32_bytes = (bh * h.n) if dom == "h" else (be * e.n)
    i32_other = (be * e.n) if dom == "h" else (bh * h.n)
    q16 = stats is not None and stats["h"][0] > 0
    if q16:
        fh, fe = format_bytes(PARAMS["n"], nhv, s, stats)
        dom_bytes = (fh * h.n) if dom == "h" else (fe * e.n)
        other_bytes = (fe * e.n) if dom == "h" else (fh * h.n)
        basis = ("compulsory bytes of the 16-bit index format the kernel reads (2 B per entry, 4 B in slices "
                 "that keep 32-bit entries, two 4-byte bases per slice and stream), weights, fields")
    else:
        dom_bytes, other_bytes = i32_bytes, i32_other
        basis = "compulsory bytes with 32-bit indices, weights, fields"
    achieved = dom_bytes / dom_t / 1e9
    kname = "k_h_stag" if dom == "h" else "k_e_stag"
    r = {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s", "frac": achieved / peak,
         "traffic": traffic_record(kname, s, dom_bytes), "kernel": kname, "peak_kind": peak_kind,
         "algorithmic_bytes_per_launch": dom_bytes, "bytes_basis": basis, "avg_launch_ms": dom_t * 1e3,
         "other_kernel_avg_launch_ms": other_t * 1e3,
         "other_kernel_achieved_gbs": other_bytes / other_t / 1e9,
         "int32_index_count": {"bytes_per_launch": i32_bytes, "achieved": i32_bytes / dom_t / 1e9,
                               "frac": i32_bytes / dom_t / 1e9 / peak,
                               "note": "the same launch counted with 32-bit indices everywhere; the kernel "
                                       "reads fewer bytes than this, so this fraction can exceed 1"}}
    if q16:
        r["index_format"] = {"name": "q16",
                             "slices_with_32bit_entries": {"h_pass": list(stats["h"][1:]),
                                                           "e_pass": list(stats["e"][1:]),
                                                           "slices": stats["h"][0]}}
    return r


def batched(M, ctx, steps, peak, peak_kind, ndom=256, nrhs=16):
    """Batched workload: 256 PEC squares and disks, node counts log-uniform in
    [2k, 60k] (about 4.3M nodes), stencil sizes n in {12, 20, 30, 40} (PHS r^3,
    largest m with 2 M_m <= n; Delta^2 HV on 31 nodes), 16 Ricker sources per
    domain, each its own right-hand side; FP32; all steps in one persistent
    cooperative launch replayed from a CUDA graph."""
    S, c = C4["courant"], C4["hv"]["c"]
    nh, alpha, k = C4["hv"]["n"], C4["hv"]["alpha"], C4["curl"]["phs_k"]
    dt, eps0, mu0, c0, eta0 = W.units(S)
    t = time.time()
    dd = C4["domains"]
    specs = W.batch_domains(ndom, dd["seed"], dd["n_min"], dd["n_max"], tuple(dd["stencils"]))
    doms, keep = [], []
    for ns, n in specs:
        nd = M.Nodes(ctx, ns.xyz, ns.period)
        st = M.Stencils(nd, nd, max(n, nh))
        cw = M.Weights(st, n, k, W.poly_degree_for(n), M.MFD_OP_GRAD)
        hw = M.Weights(st, nh, 2 * alpha + 1, 2 * alpha, M.MFD_OP_LAP_POW, alpha)
        doms.append((cw, hw, dt, eps0, mu0, -c))
        keep.append((nd, st))
    bt = M.Batch(ctx, doms, nrhs=nrhs)
    for d, (ns, n) in enumerate(specs):
        bt.set_materials(d, None, ns.pec)
        src = W.ricker_sources(ns, nrhs, C4["sources_seed0"] + d, c0, nrhs=nrhs, one_per_rhs=True)
        bt.set_sources(d, src.node, src.rhs, src.amp, src.f0, src.t0)
    setup_s = time.time() - t
    import torch
    blob0 = bt.save_state()  # t = 0: the timed run starts here again after the warm-up
    variant, variant_ms = bt.autotune(20)  # the work split, timed on this batch (state put back)
    bt.step(steps)  # captures the graph and warms up
    bt.load_state(blob0)
    del blob0
    stream = ctx.torch_stream()
    torch.cuda.synchronize()
    t0 = torch.cuda.Event(enable_timing=True)
    t1 = torch.cuda.Event(enable_timing=True)
    t0.record(stream)
    bt.step(steps)
    t1.record(stream)
    torch.cuda.synchronize()
    el = t0.elapsed_time(t1) / 1e3
    ntot = sum(ns.n for ns, _ in specs)
    upd = ntot * 3 * nrhs
    # for the comparison with the oracle: the smallest domain of each stencil size,
    # four of its right-hand sides, after the timed run (the whole step count from t = 0)
    pick = []
    for nn in sorted({n for _, n in specs}):
        cand = [d for d, (ns, n) in enumerate(specs) if n == nn]
        pick.append(min(cand, key=lambda d: specs[d][0].n))
    rhs_pick = [0, nrhs // 3, 2 * nrhs // 3, nrhs - 1]
    check = {"steps": steps, "c": c, "domains": [
        {"dom": d, "n": specs[d][1], "nodes": specs[d][0], "rhs": rhs_pick,
         "src": W.ricker_sources(specs[d][0], nrhs, 500 + d, c0, nrhs=nrhs, one_per_rhs=True),
         "ez": bt.get_field(d, M.MFD_EZ)[:, rhs_pick], "hx": bt.get_field(d, M.MFD_HX)[:, rhs_pick],
         "hy": bt.get_field(d, M.MFD_HY)[:, rhs_pick]} for d in pick]}
    byt = sum(ns.n * (4 * (max(n, 31) + n) + 4 * (4 * n + 31) + 10 * 4 * nrhs) for ns, n in specs)
    ach = byt * steps / el / 1e9
    # the L1 data path: bytes the gathers deliver to registers per step plus the stencil
    # streams once per pass, against 128 B per clock per SM. Variants 0, 1: every H-pass
    # entry of the row (L = max(n, 31)) brings Ez, Hx and Hy of all right-hand sides,
    # every E-pass curl entry Hx and Hy; variants 2, 3 (H row's HV term in the E pass):
    # every H-pass entry Ez, every E-pass entry of the row Hx and Hy
    if variant < 2:
        l1b = sum(ns.n * (max(n, 31) * 3 * 4 * nrhs + n * 2 * 4 * nrhs + 4 * (max(n, 31) + n) + 4 * (4 * n + 31))
                  for ns, n in specs)
        l1_basis = ("gathered field bytes delivered to registers (3 fields x R x 4 B per H-pass entry, "
                    "2 fields x R x 4 B per E-pass curl entry) + stencil streams once per pass")
    else:
        l1b = sum(ns.n * (max(n, 31) * 3 * 4 * nrhs + 2 * (4 * max(n, 31) + 4 * (2 * n + 31))) for ns, n in specs)
        l1_basis = ("gathered field bytes delivered to registers (Ez x R x 4 B per H-pass entry, "
                    "2 fields x R x 4 B per E-pass entry of the row) + stencil streams once per pass")
    sms = torch.cuda.get_device_properties(0).multi_processor_count
    l1_peak = sms * 128 * _sm_max_mhz() * 1e6 / 1e9
    return {"workload": f"batched {ndom} domains (squares and disks, 2k-60k nodes), {nrhs} RHS",
            "nodes": ntot, "value": upd * steps / el, "unit": UNIT, "steps": steps,
            "ms_per_step": el / steps * 1e3, "graph": bt.uses_graph, "setup_s": round(setup_s, 2),
            "autotuned": {"variant": variant,
                          "variants": ["stream prefetch, 3 blocks of 256 per SM", "no prefetch, 4 blocks per SM",
                                       "stream prefetch, H-row HV term in the E pass (H*)",
                                       "no prefetch, H-row HV term in the E pass (H*)"],
                          "ms_per_step_by_variant": [float(x) for x in variant_ms]},
            "roofline": {"bound": "hbm", "achieved": ach, "peak": peak, "unit": "GB/s", "frac": ach / peak,
                         "traffic": traffic_record("k_batch16" if variant == 0 else f"k_batch16v{variant}", 4, byt)
                         if nrhs == 16 else None,
                         "traffic_unit": "DRAM bytes per step (the persistent launch runs all steps)",
                         "kernel": f"k_batch<16, {variant}>", "peak_kind": peak_kind,
                         "algorithmic_bytes_per_step": byt},
            "l1_roofline": {"bound": "l1", "achieved": l1b * steps / el / 1e9, "peak": l1_peak, "unit": "GB/s",
                            "frac": l1b * steps / el / 1e9 / l1_peak, "bytes_per_step": l1b,
                            "peak_kind": f"nominal: {sms} SMs x 128 B per clock x the maximum SM clock",
                            "basis": l1_basis},
            "_gpu": check}


def _pec_cube(M, ctx, nx):
    """The 3D workload's node set and operators: nx^3 jittered cell-centred
    nodes in the PEC cube [0, nx]^3 (walls by images), curl stencils of 40 nodes
    (PHS r^3, degree 3) and of 44 nodes in the layer next to the walls, Delta^2
    HV on 71 nodes (r^5, degree 4), eps_r = 1 + 3 g (smoothed Gaussian random
    field), FP32 state with compensated sums, TM110 initial fields."""
    S, c, n, k, m, alpha, n_wall = (CUBE[x] for x in ("S", "c", "n", "k", "m", "alpha", "n_wall"))
    dt, eps0, mu0, c0, eta0 = W.units(S)
    t = time.time()
    nodes = W.pec_box_cells((nx, nx, nx), 0.25, 3)
    er = W.eps_r_smooth_3d(nodes.xyz, nodes.box_hi, 33)
    E0, H0 = W.tm110_fields_3d(nodes.xyz, float(nx), c0, mu0, 0.0, -0.5 * dt)
    gen_s = time.time() - t
    t = time.time()
    nd = M.Nodes(ctx, nodes.xyz, nodes.period)
    nd.set_mirror(7, nodes.box_hi)
    nhv = 2 * math.comb(2 * alpha + 3, 3) + 1
    st = M.Stencils(nd, nd, max(n_wall, nhv))
    ctx.sync()
    t_knn = time.time() - t
    t = time.time()
    sizes = M.wall_layer_sizes(nodes.xyz, nodes.box_lo, nodes.box_hi, n, n_wall)
    cw = M.Weights(st, sizes, k, m, M.MFD_OP_GRAD)
    hw = M.Weights(st, nhv, 2 * alpha + 1, 2 * alpha, M.MFD_OP_LAP_POW, alpha)
    ctx.sync()
    t_w = time.time() - t
    sim = M.Sim(ctx, 3, M.MFD_FP32, dt, eps0, mu0, -c, cw, hw, compensated=True)
    sim.set_materials(er, None)
    for comp, v in zip(range(6), (*E0, *H0)):
        sim.set_field(comp, v)
    return sim, (nd, st, cw, hw), nodes, er, np.stack(E0), np.stack(H0), {
        "generate": round(gen_s, 2), "morton_knn_images": round(t_knn, 2), "weights_fp64": round(t_w, 2),
        "curl_nodes_mean": float(sizes.mean())}


def cube3d(M, ctx, steps, peak, peak_kind, nx=200):
    """3D full-vector workload: 200^3 = 8M jittered nodes in a PEC cube, walls
    by images (every stencil among the nodes and their mirror images, image
    values signed by the parity of the field component), 2000 FP32 steps (see
    _pec_cube for the operators). Also the first step from the seeded state at
    sampled nodes (in the timed launch configuration) and a whole 32^3 run, for
    the comparison with the oracle."""
    n, alpha = CUBE["n"], CUBE["alpha"]
    nhv = 2 * math.comb(2 * alpha + 3, 3) + 1
    sim, keep, nodes, er, E0, H0, setup = _pec_cube(M, ctx, nx)
    nbar = setup["curl_nodes_mean"]  # curl entries per node (40, and 44 next to the walls)
    u0 = sim.energy()  # Eq. 20 of the initial state
    blocks3 = sim.autotune(10)  # block sizes of the two passes, timed on this cube (the state is put back)
    # the first step from the seeded initial state, before any other step
    sim.step(1)
    rng = np.random.default_rng(12)
    cell = np.floor(nodes.xyz).astype(np.int64)
    far = np.all((cell >= 12) & (cell < nx - 12), axis=1)
    corner = np.all(cell < 6, axis=1)
    ids_in = np.sort(rng.choice(np.nonzero(far)[0], 24, replace=False))
    ids_wall = np.sort(rng.choice(np.nonzero(corner)[0], 24, replace=False))
    E1 = np.stack([sim.get_field(a) for a in range(3)])
    H1 = np.stack([sim.get_field(3 + a) for a in range(3)])
    sampled = {"nx": nx, "nodes": nodes, "eps_r": er, "E0": E0, "H0": H0, "ids_in": ids_in, "ids_wall": ids_wall,
               "E1_in": E1[:, ids_in], "H1_in": H1[:, ids_in], "E1_wall": E1[:, ids_wall], "H1_wall": H1[:, ids_wall]}
    del E1, H1
    for comp in range(3):
        sim.set_field(comp, E0[comp])
        sim.set_field(3 + comp, H0[comp])
    import torch
    stream = ctx.torch_stream()
    sim.step(10)
    torch.cuda.synchronize()
    t0 = torch.cuda.Event(enable_timing=True)
    t1 = torch.cuda.Event(enable_timing=True)
    t0.record(stream)
    sim.step(steps)
    t1.record(stream)
    torch.cuda.synchronize()
    el = t0.elapsed_time(t1) / 1e3
    u_end = sim.energy()
    kk = min(steps, 100)
    ms = sim.step_timed(kk)
    small = _cube_small_gpu(M, ctx, 32, 2000)
    s4 = 4
    bh = 4 * max(nbar, nhv) + s4 * (3 * nbar + nhv) + 12 * s4
    be = 4 * nbar + s4 * 3 * nbar + 9 * s4
    h_avg, e_avg = ms[0] / kk / 1e3, ms[1] / kk / 1e3
    dom = "k_h3" if h_avg >= e_avg else "k_e3"
    dom_b = (bh if dom == "k_h3" else be) * nodes.n
    dom_t = max(h_avg, e_avg)
    ach = dom_b / dom_t / 1e9
    return {"workload": f"cube3d-pec {nx}^3 (walls by images), n={n} (44 next to the walls), N_h={nhv}, FP32",
            "autotuned_blocks": {"h_pass": blocks3[0], "e_pass": blocks3[1]}, "nodes": nodes.n,
            "value": nodes.n * 6 * steps / el, "unit": UNIT, "steps": steps, "ms_per_step": el / steps * 1e3,
            "setup_s": setup, "energy_rel_after_run": float(u_end / u0), "energy_after_steps": steps + 10,
            "roofline": {"bound": "hbm", "achieved": ach, "peak": peak, "unit": "GB/s", "frac": ach / peak,
                         "traffic": traffic_record(dom + "_images", s4, dom_b), "kernel": dom, "peak_kind": peak_kind,
                         "algorithmic_bytes_per_launch": dom_b, "avg_launch_ms": dom_t * 1e3,
                         "other_kernel_avg_launch_ms": min(h_avg, e_avg) * 1e3,
                         "step_achieved_gbs": (bh + be) * nodes.n / (el / steps) / 1e9},
            "_gpu": {"sampled": sampled, "small": small}}


CUBE = dict(S=C3["courant"], c=C3["hv"]["c"], n=C3["curl"]["n"], k=C3["curl"]["phs_k"], m=C3["curl"]["poly_m"],
            alpha=C3["hv"]["alpha"], n_wall=C3["curl"]["n_wall"])


def _cube_small_gpu(M, ctx, nx, steps):
    """The 3D workload's problem on an nx^3 PEC cube (same stencils,
    coefficients, eps_r recipe and TM110 fields), every field after `steps`
    FP32 steps."""
    sim, keep, nodes, er, E0, H0, _ = _pec_cube(M, ctx, nx)
    sim.step(steps)
    return {"nx": nx, "steps": steps, "fields": np.stack([sim.get_field(a) for a in range(6)]),
            "nodes": nodes, "eps_r": er, "E0": E0, "H0": H0}


def cavity_setup():
    """The plain method's cavity (configs/c1_cavity.json): (S_c, c, PEC box, (n, PHS k, m, alpha))."""
    nd = C1["nodes"]
    nodes = W.pec_box(tuple(nd["shape"]), nd["jitter"], nd["seed"])
    cu = C1["curl"]
    return C1["courant"], C1["hv"]["c"], nodes, (cu["n"], cu["phs_k"], cu["poly_m"], C1["hv"]["alpha"])


def cavity(M, ctx, steps=1000):
    """The plain method of the paper, FP64: 100 x 100 jittered nodes in a PEC
    square, collocated 12-node stencils (r^3, degree 2), Delta^2 HV, TM11 mode,
    CFL 0.5, 1000 steps, Ez probed at 16 nodes. L2-resident (about 9 MB per
    step): latency-bound, so only updates/s are reported. Also the relative L2
    error against the exact TM11 mode at the end."""
    S, c, nodes, (n, k, m, alpha) = cavity_setup()
    dt, eps0, mu0, c0, eta0 = W.units(S)
    nhv = 2 * math.comb(2 * alpha + 2, 2) + 1
    nd = M.Nodes(ctx, nodes.xyz, nodes.period)
    st = M.Stencils(nd, nd, max(n, nhv))
    cw = M.Weights(st, n, k, m, M.MFD_OP_GRAD)
    hw = M.Weights(st, nhv, 2 * alpha + 1, 2 * alpha, M.MFD_OP_LAP_POW, alpha)
    sim = M.Sim(ctx, 2, M.MFD_FP64, dt, eps0, mu0, -c, cw, hw)
    sim.set_materials(None, nodes.pec)
    blocks = sim.autotune(10)  # block sizes and threads per node of the two passes (the state is put back)
    ez, hx, hy = W.tm11_fields(nodes.xyz, CAV_L, c0, mu0, 0.0, -0.5 * dt)
    ez[nodes.pec == 1] = 0
    probes = W.interior_nodes(nodes, C1["probes"]["count"], C1["probes"]["seed"])
    import torch

    def run():
        sim.set_field(M.MFD_EZ, ez)
        sim.set_field(M.MFD_HX, hx)
        sim.set_field(M.MFD_HY, hy)
        sim.set_probes(probes, steps)
        stream = ctx.torch_stream()
        torch.cuda.synchronize()
        t0 = torch.cuda.Event(enable_timing=True)
        t1 = torch.cuda.Event(enable_timing=True)
        t0.record(stream)
        sim.step(steps)
        t1.record(stream)
        torch.cuda.synchronize()
        return t0.elapsed_time(t1) / 1e3

    run()
    el = run()
    T = steps * dt
    ea, xa, ya = W.tm11_fields(nodes.xyz, CAV_L, c0, mu0, T, T - 0.5 * dt)
    got = np.concatenate([sim.get_field(cc) for cc in (M.MFD_EZ, M.MFD_HX, M.MFD_HY)])
    ref = np.concatenate([ea, xa, ya])
    return {"workload": "cavity TM11, 100x100 PEC, n=12, FP64, 1000 steps", "nodes": nodes.n,
            "value": nodes.n * 3 * steps / el, "unit": UNIT, "steps": steps, "ms_per_step": el / steps * 1e3,
            "roofline": "n/a (L2-resident, latency-bound)", "autotuned_blocks": {"h_pass": blocks[0], "e_pass": blocks[1]},
            "rel_l2_vs_exact_mode": float(np.linalg.norm(got - ref) / np.linalg.norm(ref)),
            "_gpu": {"fields": got, "probes": sim.read_probes(), "steps": steps}}


def adjoint(M, ctx, steps=C5["steps"], every=C5["checkpoint_every"], l2_keep=None):
    """Differentiation workload: 500 x 500 PEC box, n = 20 (r^3, degree 2),
    Delta^2 HV, eps_r = 1 + 0.5 U, 4 Ricker sources, 8 probes, FP32, 4000
    steps: J = dt sum Ez_p^2 and dJ/deps_r, dJ/d amplitudes by the adjoint with
    checkpoints every 64 steps. Reports the forward step rate and the time of one
    gradient (forward with checkpoints + segment recomputation + adjoint), and
    of the same gradient with the whole Ez history kept on the device."""
    nodes_side = C5["nodes"]["shape"][0]
    P = _adjoint_problem(nodes_side)
    S, c, nodes = P["S"], P["c"], P["nodes"]
    dt, eps0, mu0, c0, eta0 = W.units(S)
    cw, hw, keep = _adjoint_weights(M, ctx, P)
    sim = M.Sim(ctx, 2, M.MFD_FP32, dt, eps0, mu0, -c, cw, hw, compensated=True)
    if l2_keep is not None:
        sim.set_l2_keep(l2_keep)
    eps, src, probes = P["eps"], P["src"], P["probes"]
    z = np.zeros(nodes.n)

    def setup():
        sim.set_materials(eps, nodes.pec)
        for cc in (M.MFD_EZ, M.MFD_HX, M.MFD_HY):
            sim.set_field(cc, z)
        sim.set_sources(src.node, src.amp, src.f0, src.t0)
        sim.set_probes(probes, steps)

    setup()
    sim.autotune(10)
    import torch
    stream = ctx.torch_stream()
    sim.step(steps)
    setup()
    torch.cuda.synchronize()
    t0 = torch.cuda.Event(enable_timing=True)
    t1 = torch.cuda.Event(enable_timing=True)
    t0.record(stream)
    sim.step(steps)
    t1.record(stream)
    torch.cuda.synchronize()
    fwd = t0.elapsed_time(t1) / 1e3
    peak, peak_kind = peaks()
    n_c, n_hv = P["stencil"][0], C5["hv"]["n"]
    node_b = sum(colloc_bytes(n_c, n_hv, 4))
    fwd_gbs = node_b * nodes.n * steps / fwd / 1e9
    setup()
    t = time.perf_counter()
    J, ge, ga = sim.grad(steps, every, len(src.node))
    gs = time.perf_counter() - t
    # the same gradient from the whole Ez history (4 GB here): no recomputation
    setup()
    t = time.perf_counter()
    J0, ge0, ga0 = sim.grad(steps, 0, len(src.node))
    gw = time.perf_counter() - t
    small = _adjoint_small_gpu(M, ctx)
    return {"workload": f"adjoint {nodes_side}x{nodes_side} PEC, n={P['stencil'][0]}, FP32, {steps} steps, checkpoints every {every}", "nodes": nodes.n,
            "_gpu": small,
            "forward_value": nodes.n * 3 * steps / fwd, "unit": UNIT, "forward_ms_per_step": fwd / steps * 1e3,
            "l2_keep": sim.l2_keep,
            "forward_roofline": {"bound": "hbm", "achieved": fwd_gbs, "peak": peak, "unit": "GB/s",
                                 "frac": fwd_gbs / peak, "traffic": None, "peak_kind": peak_kind,
                                 "bytes_per_node_step": node_b,
                                 "note": "whole step (H and E passes and the source/probe launch) against "
                                         "688 B per node and step (204 index, 444 weight, 40 field bytes); with "
                                         "part of the streams kept in L2 from step to step the DRAM bytes are "
                                         "fewer than these"},
            "gradient_s": gs, "gradient_over_forward": gs / fwd, "J": J,
            "grad_norm_eps": float(np.linalg.norm(ge)), "grad_amp": [float(x) for x in ga],
            "whole_history": {"gradient_s": gw, "gradient_over_forward": gw / fwd,
                              "history_bytes": (steps + 1) * nodes.n * 4,
                              "max_rel_diff_vs_checkpoints": float(np.max(np.abs(ge0 - ge)) / np.max(np.abs(ge)))}}


def _adjoint_problem(nx):
    """The differentiation workload's recipe (configs/c5_adjoint.json) on an nx x nx PEC box."""
    S, c = C5["courant"], C5["hv"]["c"]
    dt, eps0, mu0, c0, eta0 = W.units(S)
    nodes = W.pec_box((nx, nx), C5["nodes"]["jitter"], C5["nodes"]["seed"])
    er, so, pr = C5["eps_r"], C5["sources"], C5["probes"]
    cu, hv = C5["curl"], C5["hv"]
    return dict(S=S, c=c, nodes=nodes, eps=W.eps_r_uniform(nodes.n, er["seed"], er["lo"], er["span"]),
                src=W.ricker_sources(nodes, so["count"], so["seed"], c0),
                probes=W.interior_nodes(nodes, pr["count"], pr["seed"]),
                stencil=(cu["n"], cu["phs_k"], cu["poly_m"], hv["n"], hv["alpha"]))


def _adjoint_weights(M, ctx, P):
    n, k, m, nh, alpha = P["stencil"]
    ns = P["nodes"]
    nd = M.Nodes(ctx, ns.xyz, ns.period)
    st = M.Stencils(nd, nd, max(n, nh))
    cw = M.Weights(st, n, k, m, M.MFD_OP_GRAD)
    hw = M.Weights(st, nh, 2 * alpha + 1, 2 * alpha, M.MFD_OP_LAP_POW, alpha)
    return cw, hw, (nd, st)


def _adjoint_small_gpu(M, ctx, nx=60, steps=400):
    """J and its gradient (FP32, whole Ez history) on a reduced 60 x 60 box for the oracle's adjoint."""
    P = _adjoint_problem(nx)
    dt, eps0, mu0, c0, eta0 = W.units(P["S"])
    ns = P["nodes"]
    cw, hw, keep = _adjoint_weights(M, ctx, P)
    sim = M.Sim(ctx, 2, M.MFD_FP32, dt, eps0, mu0, -P["c"], cw, hw, compensated=True)
    sim.set_materials(P["eps"], ns.pec)
    z = np.zeros(ns.n)
    for cc in (M.MFD_EZ, M.MFD_HX, M.MFD_HY):
        sim.set_field(cc, z)
    src = P["src"]
    sim.set_sources(src.node, src.amp, src.f0, src.t0)
    sim.set_probes(P["probes"], steps)
    J, ge, ga = sim.grad(steps, 0, len(src.node))
    return {"nx": nx, "steps": steps, "J": J, "g_eps": ge, "g_amp": ga}


def yee(M, ctx, peak, peak_kind, big=8192, steps=1000, nx=1000, pulse_steps=5000, stride=4):
    """The FDTD (Yee) reference scheme (Eq. 5) on the GPU, FP32:
    (a) throughput and HBM roofline of the fused step kernel on a big x big
        periodic grid (compulsory bytes: Ez, Hx, Hy read and written once,
        24 B per cell and step), random fields;
    (b) the pulse workload's problem on an nx x nx grid (carrier 12 h, S = 0.5,
        pulse_steps steps): updates/s next to the meshless step, and the phase
        speed at the carrier measured on row nx/2 (Sec. 6 analysis) against
        Eq. 6 and the physical speed."""
    import math
    import torch
    S = PARAMS["S"]
    dt, eps0, mu0, c0, eta0 = W.units(S)
    out = {}
    y = M.Yee(ctx, big, big, M.MFD_FP32, dt, 1.0, eps0, mu0)
    rng = np.random.default_rng(1)
    for comp in (M.MFD_EZ, M.MFD_HX, M.MFD_HY):
        y.set_field(comp, rng.standard_normal((big, big)))
    y.step(64)
    stream = ctx.torch_stream()
    torch.cuda.synchronize()
    t0 = torch.cuda.Event(enable_timing=True)
    t1 = torch.cuda.Event(enable_timing=True)
    t0.record(stream)
    y.step(steps)
    t1.record(stream)
    torch.cuda.synchronize()
    el = t0.elapsed_time(t1) / 1e3
    k = min(steps, 200)
    spl = y.steps_per_launch  # steps fused per launch (no sources or probes here)
    ms = y.step_timed(k) / k * spl  # per launch
    cells = big * big
    alg = 24.0 * cells  # Ez, Hx, Hy read and written once per launch
    out["grid"] = {"cells": cells, "steps": steps, "ms_per_step": el / steps * 1e3,
                   "value": 3 * cells * steps / el, "unit": UNIT, "steps_per_launch": spl,
                   "roofline": {"bound": "hbm", "achieved": alg / (ms / 1e3) / 1e9, "peak": peak, "unit": "GB/s",
                                "frac": alg / (ms / 1e3) / 1e9 / peak,
                                "traffic": traffic_record(f"k_yee{spl}_{big}", 4, alg),
                                "kernel": f"k_yee<float, S={spl}>",
                                "peak_kind": peak_kind, "algorithmic_bytes_per_launch": alg,
                                "avg_launch_ms": ms}}
    # one step per launch (a probe forces it; k_yee_post records the probe after each step)
    y.set_probes(np.array([0]), steps)
    y.step(8)
    torch.cuda.synchronize()
    t0.record(stream)
    y.step(steps)
    t1.record(stream)
    torch.cuda.synchronize()
    el1 = t0.elapsed_time(t1) / 1e3
    ms1 = y.step_timed(k) / k
    out["grid_one_step"] = {"cells": cells, "steps": steps, "ms_per_step": el1 / steps * 1e3,
                            "value": 3 * cells * steps / el1, "unit": UNIT, "steps_per_launch": 1,
                            "roofline": {"bound": "hbm", "achieved": alg / (ms1 / 1e3) / 1e9, "peak": peak,
                                         "unit": "GB/s", "frac": alg / (ms1 / 1e3) / 1e9 / peak,
                                         "traffic": traffic_record(f"k_yee1_{big}", 4, alg),
                                         "kernel": "k_yee<float, S=1> (+ k_yee_post)", "peak_kind": peak_kind,
                                         "algorithmic_bytes_per_launch": alg, "avg_launch_ms": ms1}}
    del y
    lam = PARAMS["wavelength"]
    g = np.arange(nx, dtype=float)
    xy = np.stack(np.meshgrid(g, g), -1).reshape(-1, 2)
    for tag, direction, x0, line, h_line, phi in (
            ("pulse", (1, 0), nx / 2, np.arange(nx) + (nx // 2) * nx, 1.0, 0.0),
            ("pulse_45", (1, 1), nx / math.sqrt(2) / 2, np.arange(nx) * (nx + 1), math.sqrt(2), math.pi / 4)):
        y = M.Yee(ctx, nx, nx, M.MFD_FP32, dt, 1.0, eps0, mu0)
        ez, _, _ = W.gaussian_pulse(xy, nx, x0, 2 * lam, c0, eta0, dt, lam, direction=direction)
        _, hx, _ = W.gaussian_pulse(xy + np.array([0.0, 0.5]), nx, x0, 2 * lam, c0, eta0, dt, lam,
                                    direction=direction)  # Hx at (i, j + 1/2)
        _, _, hy = W.gaussian_pulse(xy + np.array([0.5, 0.0]), nx, x0, 2 * lam, c0, eta0, dt, lam,
                                    direction=direction)  # Hy at (i + 1/2, j)
        y.set_field(M.MFD_EZ, ez)
        y.set_field(M.MFD_HX, hx)
        y.set_field(M.MFD_HY, hy)
        y.set_probes(line, pulse_steps)
        torch.cuda.synchronize()
        t0.record(stream)
        y.step(pulse_steps)
        t1.record(stream)
        torch.cuda.synchronize()
        el = t0.elapsed_time(t1) / 1e3
        nt = pulse_steps // stride
        samples = y.read_probes()[stride - 1::stride]
        spec, kidx, c, _ = M.dispersion(ctx, samples, h_line, stride * dt, c0, 1)
        rep = _ridge_report(M, spec, kidx, c, nt, stride * dt, phi, el, 0.0, stride, h_line)
        out[tag] = {"cells": nx * nx, "steps": pulse_steps, "ms_per_step": el / pulse_steps * 1e3,
                    "value": 3 * nx * nx * pulse_steps / el, "unit": UNIT,
                    "l2_note": "24 MB state: L2-resident, launch/latency bound",
                    "carrier": rep["carrier"], "band_j": rep["band_j"], "err_l1": rep["err_l1"],
                    "eq6_err_l1": rep["fdtd_err_l1"]}
        del y
    return out


def hv_search(M, ctx, nx=200, steps=10000, ncand=16, rounds=2):
    """The hyperviscosity coefficient search (mfd_hv_search) on the setup of
    Sec. 6: a periodic jittered 200 x 200 layout, Courant number 1/(10 sqrt 2),
    a sigma = 2 h Gaussian pulse, alpha = 2, here with n = 30 (PHS r^5,
    monomials to degree 4), 10,000 steps per round, ncand candidates per round
    in [1e-6, 1e-1], energy checked every 100 steps against 1 % growth."""
    import math
    S = 1 / (10 * math.sqrt(2))
    dt, eps0, mu0, c0, eta0 = W.units(S)
    nodes = W.periodic_box((nx, nx), 0.25, 6)
    nd = M.Nodes(ctx, nodes.xyz, nodes.period)
    st = M.Stencils(nd, nd, 31)
    cw = M.Weights(st, 30, 5, 4, M.MFD_OP_GRAD)
    hw = M.Weights(st, 31, 5, 4, M.MFD_OP_LAP_POW, 2)
    ez, hx, hy = W.gaussian_pulse(nodes.xyz, nx, nx / 2, 2.0, c0, eta0, dt, None)
    t0 = time.perf_counter()
    c, hist = M.hv_search(ctx, cw, hw, dt, eps0, mu0, ez, hx, hy, -6.0, -1.0, ncand=ncand, rounds=rounds,
                          nsteps=steps, check_every=100, tol=0.01)
    el = time.perf_counter() - t0
    updates = nodes.n * 3 * ncand * steps * rounds
    last = hist[-1]
    k = int(np.argmin(np.abs(last[:, 0] - math.log10(c))))
    return {"workload": f"hv-search periodic {nx}x{nx}, S=1/(10 sqrt 2), sigma=2, n=30, alpha=2",
            "nodes": int(nodes.n), "candidates_per_round": ncand, "rounds": rounds, "steps_per_round": steps,
            "log10_c": math.log10(c), "u_max_at_c": float(last[k, 1]), "u_end_at_c": float(last[k, 2]),
            "final_interval_log10": 5.0 / ncand ** rounds,
            "seconds": el, "value": updates / el, "unit": UNIT,
            "paper_log10_c_context": -4.76}


def _line_analysis(M, sim, steps, stride, h_line, phi):
    """Runs `steps` steps with the line's probes set and analyses them (Sec. 6):
    c(w) at the carrier and the l1 error of Eq. 26 over the band where the
    spectrum is present (rows whose largest component is >= 1 % of the overall
    largest), next to the Yee scheme's phase speed (Eq. 6) at angle phi."""
    import math
    S = PARAMS["S"]
    dt, eps0, mu0, c0, eta0 = W.units(S)
    t0 = time.perf_counter()
    sim.step(steps)
    sim.ctx.sync()
    t_run = time.perf_counter() - t0
    nt = steps // stride
    dts = stride * dt
    t0 = time.perf_counter()
    sim.dispersion(stride, nt, h_line, c0, 1, spectrum=False)
    t_an = time.perf_counter() - t0
    spec, kidx, c, _ = sim.dispersion(stride, nt, h_line, c0, 1)
    return _ridge_report(M, spec, kidx, c, nt, dts, phi, t_run, t_an, stride, h_line)


def _ridge_report(M, spec, kidx, c, nt, dts, phi, t_run, t_an, stride, h_line):
    """c(w) at the carrier, and Eq. 25-26 summed over the band of the pulse:
    the contiguous rows around the carrier's row (positive frequencies,
    j < nt / 2; a real signal mirrors them at nt - j) whose largest component
    is >= 1 % of the carrier row's. The Yee phase speed (Eq. 6) at the same
    frequencies and angle for comparison."""
    import math
    S = PARAMS["S"]
    dt, eps0, mu0, c0, eta0 = W.units(S)
    rowmax = spec.max(axis=1)
    w0 = c0 * 2 * math.pi / PARAMS["wavelength"]  # carrier angular frequency (per dt)
    j0 = int(round(w0 * nt * dts / (2 * math.pi)))
    lo = hi = j0
    while lo > 1 and rowmax[lo - 1] >= 1e-2 * rowmax[j0]:
        lo -= 1
    while hi + 1 < (nt + 1) // 2 and rowmax[hi + 1] >= 1e-2 * rowmax[j0]:
        hi += 1
    band = range(lo, hi + 1)
    fd = {j: M.fdtd_phase_speed(2 * math.pi * j / (nt * dts) * dt, S, phi) for j in band}
    return {"samples": nt, "stride": stride, "h_line": h_line, "run_s": t_run, "analysis_ms": t_an * 1e3,
            "carrier": {"j": j0, "k_index": int(kidx[j0]), "c": float(c[j0]), "rel_err": float(abs(c[j0] - c0) / c0),
                        "fdtd_c": fd[j0], "fdtd_rel_err": abs(fd[j0] - c0) / c0},
            "band_j": [lo, hi], "err_l1": float(sum(abs(c[j] - c0) for j in band)),
            "fdtd_err_l1": float(sum(abs(fd[j] - c0) for j in band))}


def dispersion(M, ctx, wts, e, reset, comp, steps=5000, stride=4):
    """Phase speed of the pulse workload against the physical one (Sec. 6,
    Eqs. 24-26), analysed on the GPU (mfd_sim_dispersion): at 0 degrees on the
    equispaced seed line y = L/2 of the E set, and at 45 degrees (Eq. 27: the
    same modulated pulse along the diagonal) on an E set whose diagonal x = y
    is equispaced (spacing sqrt 2), each with every node of the line a probe."""
    import math
    nx = int(round(e.period[0]))
    lam = PARAMS["wavelength"]
    dt, eps0, mu0, c0, eta0 = W.units(PARAMS["S"])
    line = np.nonzero(e.xyz[:, 1] == nx // 2)[0]
    line = line[np.argsort(e.xyz[line, 0])]
    sim = make_sim(M, ctx, wts, M.MFD_FP32, comp)
    reset(sim, 8)
    sim.set_probes(line, steps)
    out = {"c0": c0, "steps": steps, "line_nodes": int(len(line)),
           "phi_0": _line_analysis(M, sim, steps, stride, 1.0, 0.0)}
    del sim
    # 45 degrees: the E set with an equispaced diagonal, the H set as before
    e45 = W.periodic_box((nx, nx), 0.25, 2, seed_diagonal=True)
    h45 = W.periodic_box((nx, nx), 0.25, 3, offset=(0.5, 0.5))
    wts45, _, _ = build_weights(M, ctx, e45, h45)
    sim = make_sim(M, ctx, wts45, M.MFD_FP32, comp)
    x0 = nx / math.sqrt(2) / 2
    ez, _, _ = W.gaussian_pulse(e45.xyz, nx, x0, 2 * lam, c0, eta0, dt, lam, direction=(1, 1))
    _, hx, hy = W.gaussian_pulse(h45.xyz, nx, x0, 2 * lam, c0, eta0, dt, lam, direction=(1, 1))
    for comp_, v in ((M.MFD_EZ, ez), (M.MFD_HX, hx), (M.MFD_HY, hy)):
        sim.set_field(comp_, v)
    diag = np.nonzero(e45.xyz[:, 0] == e45.xyz[:, 1])[0]
    diag = diag[np.argsort(e45.xyz[diag, 0])]
    sim.set_probes(diag, steps)
    out["phi_45"] = _line_analysis(M, sim, steps, stride, math.sqrt(2), math.pi / 4)
    del sim, wts45
    return out


def pulse_reduced_gpu(M, ctx, nx=160, steps=5000, every=100):
    """The headline workload's problem on an nx x nx + nx x nx staggered periodic
    square (same stencils, coefficients and pulse), stepped on the GPU for the
    full step count in FP32 (compensated and plain sums) and FP64: all fields
    after every `every` steps and the probe series, kept for the comparison
    with the oracle (oracle_checks)."""
    e, h = node_sets(nx)
    wts, _, _ = build_weights(M, ctx, e, h)
    dt = W.units(PARAMS["S"])[0]
    ez, hx, hy = pulse_fields(e, h, nx, dt)
    probes = W.interior_nodes(e, 16, 24)
    out = {"nx": nx, "steps": steps, "every": every}
    for tag, prec, comp in (("fp32_compensated", M.MFD_FP32, True), ("fp32_plain", M.MFD_FP32, False),
                            ("fp64", M.MFD_FP64, False)):
        sim = make_sim(M, ctx, wts, prec, comp)
        for c_, v in ((M.MFD_EZ, ez), (M.MFD_HX, hx), (M.MFD_HY, hy)):
            sim.set_field(c_, v)
        sim.set_probes(probes, steps)
        snaps = []
        for _ in range(steps // every):
            sim.step(every)
            snaps.append(np.concatenate([sim.get_field(c_) for c_ in (M.MFD_EZ, M.MFD_HX, M.MFD_HY)]))
        out[tag] = {"snaps": snaps, "probes": sim.read_probes()}
        del sim
    return out


def accuracy(M, ctx, wts, steps, reset):
    """FP32 (compensated and plain) against FP64, all on the GPU, after `steps` steps:
    relative L2 error of all fields together and the largest absolute error."""
    fields = {}
    for tag, prec, comp in (("fp64", M.MFD_FP64, False), ("fp32_compensated", M.MFD_FP32, True),
                            ("fp32_plain", M.MFD_FP32, False)):
        sim = make_sim(M, ctx, wts, prec, comp)
        reset(sim, steps)
        sim.step(steps)
        fields[tag] = np.concatenate([sim.get_field(c) for c in (M.MFD_EZ, M.MFD_HX, M.MFD_HY)])
        fields[tag + "_probes"] = sim.read_probes()
        del sim
    ref = fields["fp64"]
    out = {"steps": steps}
    for tag in ("fp32_compensated", "fp32_plain"):
        d = fields[tag] - ref
        pd = fields[tag + "_probes"] - fields["fp64_probes"]
        out[tag] = {"rel_l2": float(np.linalg.norm(d) / np.linalg.norm(ref)), "max_abs": float(np.max(np.abs(d))),
                    "probe_rel_l2": float(np.linalg.norm(pd) / np.linalg.norm(fields["fp64_probes"]))}
    return out


if __name__ == "__main__":
    main()
