#!/usr/bin/env python
"""Throughput and latency of the single-layer dual-mesh BEM hot path on GB300.

One step = one full pass of the hot path for one request: assemble the operator
(triangle-pair fill of L^A, L^phi, Kbar with BC sources, singular corrections,
the layered-medium tables and reflected fill in a stratified background, Gram
I_x, Y11/Y21 by LU), build the plane-wave right-hand side and solve by GMRES to
the stated relative residual (plus the bistatic RCS in a homogeneous
background).  Workloads with a frequency sweep take the next frequency of the
sweep at every step.  The metric is solves/s (and p50/p99 latency per solve) at
that residual.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference] [--workload NAME]

Under torchrun (N > 1) every rank runs independent replicas (the path has no
exchange step); value = solves of all ranks / max time over ranks.
"""
from __future__ import annotations

import argparse
import json
import os
import platform
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

from workloads.meshes import box, copper_wire, cylinder_array, icosphere  # noqa: E402

# ----------------------------------------------------------------------------- workloads
WORKLOADS = {
    # Dielectric sphere in free space, icosphere sub 2, plain method in complex FP64
    "sphere-r0.1-epsr4-sub2-300MHz-fp64": dict(
        mesh=lambda: icosphere(2, 0.1), obj=None, mats=[(4.0, 1.0, 0.0)], bg=(1.0, 1.0, 0.0, 0.0), freq=300e6,
        precision=0, tol=1e-8, khat=[0.0, 0.0, -1.0], pol=[1.0, 0.0, 0.0], n_angles=181),
}
# n x n dielectric cylinders (eps_r 6, r 120 nm, h 300 nm, period 500 nm, 240 triangles
# each) in free space at 1 um, complex FP32 operator (FP64 singular terms), one plane
# wave at normal incidence, GMRES with FP64-residual iterative refinement to 1e-8.  8 x 8: 15,360 triangles, N = 61,376; 4 x 4 is the small
# case kept for profiling captures (global blocks 383 MB, above the L2 size).
for _n in (8, 4):
    WORKLOADS[f"metasurface-{_n}x{_n}-cyl-epsr6-1um-freespace-c64"] = dict(
        mesh=(lambda n=_n: cylinder_array(n, n, 120e-9, 300e-9, 500e-9)[:2]), obj=("array", _n),
        mats=[(6.0, 1.0, 0.0)] * (_n * _n), bg=(1.0, 1.0, 0.0, 0.0), freq=299792458.0 / 1e-6, precision=1,
        tol=1e-8, khat=[0.0, 0.0, -1.0], pol=[1.0, 0.0, 0.0], n_angles=181)
# The 8 x 8 metasurface under 8 plane waves per request (incidence 0 - 17.5 deg in
# 2.5 deg steps in the xz plane, TE and TM alternating), solved together: one
# assembly and one lockstep 8-RHS GMRES per step; every right-hand side counts as
# a solve.
# (4 x 4: the small case kept for profiling captures of the several-RHS kernels.)
_TH8 = np.radians(2.5 * np.arange(8))
for _n in (8, 4):
    WORKLOADS[f"metasurface-{_n}x{_n}-cyl-epsr6-1um-freespace-c64-8angles"] = dict(
        WORKLOADS[f"metasurface-{_n}x{_n}-cyl-epsr6-1um-freespace-c64"],
        khat=[[float(np.sin(t)), 0.0, -float(np.cos(t))] for t in _TH8],
        pol=[[0.0, 1.0, 0.0] if i % 2 == 0 else [float(np.cos(t)), 0.0, float(np.sin(t))] for i, t in enumerate(_TH8)],
        n_angles=181, e2e_steps=3)
# The same metasurfaces with the FP64-accurate refinement residual (complex64
# operator + low parts of an FP64 fill): solutions converge to the FP64 system.
for _n in (8, 4):
    for _sfx in ("", "-8angles"):
        WORKLOADS[f"metasurface-{_n}x{_n}-cyl-epsr6-1um-freespace-c64x2{_sfx}"] = dict(
            WORKLOADS[f"metasurface-{_n}x{_n}-cyl-epsr6-1um-freespace-c64{_sfx}"], precision=2)
# The 8 x 8 metasurface in free space under 32 plane waves per request (incidence
# 0 - 77.5 deg in 2.5 deg steps in the xz plane, TE and TM alternating), complex64
# operator with the FP64-accurate refinement residual, GMRES to 1e-8 of the FP64
# system, 181-angle RCS per plane wave.  4 x 4: the profiling case.
_TH32 = np.radians(2.5 * np.arange(32))
for _n in (8, 4):
    for _p, _sfx in ((2, "c64x2"), (1, "c64")):
        WORKLOADS[f"metasurface-{_n}x{_n}-cyl-epsr6-1um-freespace-{_sfx}-32angles"] = dict(
            WORKLOADS[f"metasurface-{_n}x{_n}-cyl-epsr6-1um-freespace-c64"], precision=_p,
            khat=[[float(np.sin(t)), 0.0, -float(np.cos(t))] for t in _TH32],
            pol=[[0.0, 1.0, 0.0] if i % 2 == 0 else [float(np.cos(t)), 0.0, float(np.sin(t))]
                 for i, t in enumerate(_TH32)],
            n_angles=181, e2e_steps=3)
# The paper-shaped case: the same 8 x 8 cylinders resting on a glass half-space
# (eps_r 2.25 below z = 0, air above), 32 plane waves from the air side through the
# interface (incidence 0 - 77.5 deg, TE/TM alternating), complex64 operator with the
# FP64-accurate refinement residual, GMRES to 1e-8 of the FP64 system, then the
# bistatic RCS of each plane wave at 90 directions of the upper half-space
# (theta 0 - 89 deg, phi = 0; reciprocity with the stack's plane waves).  4 x 4:
# the profiling case.
for _n in (8, 4):
    for _p, _sfx in ((2, "c64x2"), (1, "c64")):
        WORKLOADS[f"metasurface-{_n}x{_n}-cyl-epsr6-1um-onglass-{_sfx}-32angles"] = dict(
            WORKLOADS[f"metasurface-{_n}x{_n}-cyl-epsr6-1um-freespace-{_sfx}-32angles"],
            mats=[(6.0, 1.0, 0.0, 0)] * (_n * _n), layers=[(1.0, 1.0, 0.0, 0.0), (2.25, 1.0, 0.0, 0.0)], z_top=0.0,
            bottom="halfspace", n_angles=90, rcs_theta_max_deg=89.0)
# Multiscale conductor in a layered substrate: a copper bar (sigma 5.8e7 S/m,
# 100 x 2 x 1 um, 2,048 graded triangles, N = 8,191) in the middle of a 10 um SiO2
# layer (eps_r 3.9) over 200 um of Si (eps_r 11.9, sigma 10 S/m) over a PEC ground,
# air above; normally incident plane wave through the stack, polarised along the
# bar; 20 log-spaced frequencies 1 MHz - 50 GHz (one per step), complex FP64.
WIRE_FREQS = [float(f) for f in np.logspace(6.0, np.log10(50e9), 20)]
WORKLOADS["copper-wire-sio2-si-pec-1MHz-50GHz-fp64"] = dict(
    mesh=copper_wire, obj=None, mats=[(1.0, 1.0, 5.8e7, 1)],
    layers=[(1.0, 1.0, 0.0, 0.0), (3.9, 1.0, 0.0, 10e-6), (11.9, 1.0, 10.0, 200e-6)], z_top=0.0, bottom="pec",
    freqs=WIRE_FREQS, precision=0, tol=1e-8, maxit=6000, khat=[0.0, 0.0, -1.0], pol=[1.0, 0.0, 0.0], n_angles=0,
    e2e_steps=20)
# Serving with continuous batching (scaled to sizes the direct Y solve serves): a seeded
# catalogue of 16 models (4 spheres and 4 ellipsoids, icosphere sub 1 or 2, semi-axes
# U[0.05, 0.2] m, eps_r U[2, 12], loss tangent U[0, 0.02]; each in free space and
# 1.2 semi-axes above a 3-layer ground: air / 5 cm slab eps_r 4 / half-space eps_r 10,
# sigma 0.01 S/m) x 16 frequency bins (k0 a_max log-uniform 0.1 - 2), i.e. 256 cache
# keys; requests arrive as a Poisson stream of 200 per second (200 per step), each
# drawing its key from a Zipf(1.1) popularity over the keys (so keys repeat), 1 - 16
# plane waves (incidence U[0, 70] deg, azimuth uniform, TE or TM), tolerance 1e-8.
# Served by 2 workers, lockstep batches of up to 32 right-hand sides, complex64
# operators with the FP64-accurate residual, a 150 GB operator cache; the plain FP64
# single-solve path (one right-hand side per solve, one worker) replays one step's
# trace for comparison.
WORKLOADS["serving-catalogue-poisson200-c64x2"] = dict(
    kind="serving", n_models=16, n_freqs=16, rate=200.0, requests=200, zipf=1.1, nrhs_max=16, tol=1e-8,
    workers=2, max_batch=32, precision=2, budget=150 << 30, khat=[0.0, 0.0, -1.0], pol=[1.0, 0.0, 0.0],
    mesh=lambda: icosphere(1, 0.1), obj=None, mats=[(4.0, 1.0, 0.0)], bg=(1.0, 1.0, 0.0, 0.0), freq=300e6,
    n_angles=0)
# Batched mixed-precision frequency sweep over uneven instances: 8 seeded
# instances (7 spheres/ellipsoids, icosphere sub 2 or 3, semi-axes U[0.05, 0.2] m,
# eps_r U[2, 12], loss tangent U[0, 0.02]; one sub-4 sphere of 0.1 m, eps_r 4) in
# free space, 16 log-spaced frequencies each from k0 a_max = 0.01 to where
# sqrt(eps_r) k0 h_mean = 2 pi / 10, 8 plane waves per frequency (incidence
# (i + 1/2) 22.5 deg, phi = 0, theta-polarised); complex64 operators (FP64
# singular terms), products on the tensor cores from the measured crossover,
# refinement to 1e-8.  One step = the whole sweep (128 assemblies, 1,024 solves)
# through the serving loop with an emptied cache: 2 workers overlap the
# operators; the same sweep on one worker is reported beside it.
WORKLOADS["sweep-8instances-16freqs-8angles-c64"] = dict(
    kind="sweep", n_inst=8, n_freqs=16, n_angles_inc=8, tol=1e-8, workers=2, max_batch=8, precision=1,
    budget=150 << 30, khat=[0.0, 0.0, -1.0], pol=[1.0, 0.0, 0.0],
    mesh=lambda: icosphere(1, 0.1), obj=None, mats=[(4.0, 1.0, 0.0)], bg=(1.0, 1.0, 0.0, 0.0), freq=300e6,
    n_angles=0)
# Delta-gap port (Sec. IV-B, the antenna alone over the ground): the half-wave
# dipole of the sphere-array experiment, a 75 x 750 x 37.5 mm prism centred at
# (0, 0, 493.75 mm) (4 x 32 x 2 cells, 800 triangles), over the ground of Table I
# (sphere-array column: air above z = 375 mm; 525 mm of eps_r 3.47, 1.725 mS/m;
# half-space eps_r 6.5, 3.338 mS/m below z = -150 mm), driven by a delta-gap edge
# port at its centre (the ring in the plane y = 0); S11 against 50 ohm at 16
# frequencies 150 - 250 MHz, one per step (assemble, port right-hand side, GMRES
# to 1e-8, port current, S11), complex FP64.  The prism is a lossy metal of 1e3
# S/m (skin depth 1.1 mm at 200 MHz): the skin-depth splitting of the internal
# kernel caps a source triangle at 4,096 children, which copper (5.8e7 S/m, skin
# depth 4.7 um) would exceed by orders of magnitude at 2 cm cells.
WORKLOADS["dipole-tableI-ground-port-s11-150-250MHz-fp64"] = dict(
    mesh=lambda: box(0.075, 0.75, 0.0375, 4, 32, 2, center=(0.0, 0.0, 0.49375)), obj=None,
    mats=[(1.0, 1.0, 1e3, 0)],
    layers=[(1.0, 1.0, 0.0, 0.0), (3.47, 1.0, 0.001725, 0.525), (6.5, 1.0, 0.003338, 0.0)], z_top=0.375,
    bottom="halfspace", freqs=[float(f) for f in np.linspace(150e6, 250e6, 16)], precision=0, tol=1e-8,
    ports=[(0, (0.0, 1.0, 0.0), 0.0)], z0=50.0, khat=[0.0, 0.0, -1.0], pol=[1.0, 0.0, 0.0], n_angles=0,
    e2e_steps=4)
DEFAULT_WORKLOAD = "metasurface-8x8-cyl-epsr6-1um-onglass-c64x2-32angles"


def _nrhs(W):
    """Right-hand sides per step: one per port, else one per plane wave."""
    return len(W["ports"]) if "ports" in W else len(np.atleast_2d(W["khat"]))


def _freqs(W):
    return W.get("freqs") or [W["freq"]]


def _stack(sldm, W):
    if "layers" in W:
        return sldm.Stack(W["layers"], z_top=W["z_top"],
                          bottom=sldm.BOTTOM_PEC if W["bottom"] == "pec" else sldm.BOTTOM_HALFSPACE)
    return sldm.Stack([W["bg"]])


def _obj_ids(W):
    if isinstance(W["obj"], tuple) and W["obj"][0] == "array":
        n = W["obj"][1]
        return cylinder_array(n, n, 120e-9, 300e-9, 500e-9)[2]
    return W["obj"]

L2_FLUSH_BYTES = 512 << 20  # larger than the 129 MB L2

# Roofline denominators: MEASURED_PEAKS.json when present, else the recorded
# fallback measurement.  ALU peaks derive from unit counts x maximum SM clock:
# FP64: 152 SMs x 2 FMA x 2 flop x 2.07 GHz (1.26 TFLOP/s, the part's nominal 1.25).
FALLBACK_HBM_GBS = 6800.0
FP64_PEAK_TFLOPS = 152 * 2 * 2 * 2.07e9 / 1e12
# Fill rooflines, in Green's-function evaluations per second (36 per triangle pair).
# FP32 fill: bound by the special-function unit, 16 operations per SM per clock,
# three per evaluation of a lossless kernel (1/R, sin and cos of k R; a lossy
# kernel adds exp):  152 x 16 x 2.07 GHz / 3.
# FP64 fill: bound by the FP64 pipe (2 FMA-pipe operations per SM per clock on
# this part) with FP64_OPS_PER_EVAL pipe operations per evaluation, the count of
# fill_L_bulk<double> as ncu reports it (DFMA + DMUL + DADD per evaluation).
SFU_OPS_PER_S = 152 * 16 * 2.07e9
FILL_F32_PEAK_EVALS = SFU_OPS_PER_S / 3.0
FP64_OPS_PER_S = 152 * 2 * 2.07e9
FP64_OPS_PER_EVAL = 43.0
FILL_F64_PEAK_EVALS = FP64_OPS_PER_S / FP64_OPS_PER_EVAL
# The reflected (layered) fill in FP64: images, static z-rho images and a bilinear
# remainder lookup per evaluation; FP64 pipe operations per evaluation from ncu's
# DFMA + DMUL + DADD counts of fill_reflected_kernel<double2> on the 4 x 4 glass case.
FP64_OPS_PER_EVAL_REFL = 292.0


# DRAM traffic per algorithmic byte of the HBM-streaming main product stage, from
# one ncu capture of the kernel (dram__bytes_read.sum + dram__bytes_write.sum of
# the gemv_main launch, 4 x 4 metasurface, 423,936,000 algorithmic bytes per
# launch), valid while that kernel's source is unchanged (sha256 prefix of its
# text in csrc/<file>); for any other source the line reports traffic null.
GEMV_TRAFFIC = {
    # main-stage launch of the 4 x 4 metasurface, 32 right-hand sides (profiles/gemm_tc_metasurface-4x4-32angles-c64x2.md)
    "gemm_tc_kernel": dict(sha="78e503ea925c5ae5", file="gemm_tc.cu",
                           per_alg_byte=(450.872235e6 + 7.982507e6) / 423.936e6),
}


def kernel_sha(name, file="dense.cu"):
    """sha256 prefix of a kernel's definition in csrc/<file> (its template or attribute line to the closing brace)."""
    import hashlib
    s = open(os.path.join(ROOT, "paper_2106_06184_gb300", "csrc", file)).read()
    i = s.index(" " + name + "(")
    a = s.rindex("__global__", 0, i)
    t = s.rfind("template <", 0, i)
    if t >= 0 and t > s.rfind("}", 0, a):
        a = t
    depth, j = 0, s.index("{", i)
    while True:
        depth += {"{": 1, "}": -1}.get(s[j], 0)
        if depth == 0:
            break
        j += 1
    return hashlib.sha256(s[a:j + 1].encode()).hexdigest()[:16]


NESTED_MIN = 2500  # order of M_l from which an FP64 operator applies Y E by inner solves (library default)


def lu_flops(obj_sizes, precision=0):
    """Real flops of the FP64 batched direct solves of one assembly: per object the
    LU of M_l (n = N_e^o + N_t^o - 1) with its N_e^o right-hand sides (not for the
    objects of an FP64 operator at or above NESTED_MIN, whose Y E comes from inner
    solves), and the inverse of the preconditioner's Schur complement (n = N_t^o - 1,
    n right-hand sides).  Complex LU: n^3/3 multiply-adds; forward plus back
    substitution: n^2 per right-hand side; 8 real flops per complex multiply-add."""
    f = 0.0
    for ne_o, nt_o in obj_sizes:
        sys = [(nt_o - 1, nt_o - 1)]
        if not (precision == 0 and ne_o + nt_o - 1 >= NESTED_MIN):
            sys.append((ne_o + nt_o - 1, ne_o))
        for n, r in sys:
            f += 8.0 * (n ** 3 / 3.0 + n * n * r)
    return f


def peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        try:
            d = json.load(open(p))
            return float(d.get("hbm_gbs", FALLBACK_HBM_GBS)), "measured"
        except Exception:
            pass
    return FALLBACK_HBM_GBS, "fallback"


# ----------------------------------------------------------------------------- clocks
class ClockSampler:
    """nvidia-smi samples during the timed region (SM clock and throttle reasons)."""

    Q = ("clocks.sm,clocks.max.sm,clocks_event_reasons.active,clocks_event_reasons.hw_slowdown,"
         "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
         "clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index, self.rows, self.proc = index, [], None

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.Q}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except Exception:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.rows.append([c.strip() for c in line.split(",")])

    def stop(self):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()
        sm = [float(r[0]) for r in self.rows if r and r[0].replace(".", "").isdigit()]
        mx = [float(r[1]) for r in self.rows if len(r) > 1 and r[1].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = set()
        for r in self.rows:
            for k, n in enumerate(names):
                if len(r) > 3 + k and r[3 + k].lower() == "active":
                    reasons.add(n)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": sorted(reasons), "samples": len(sm)}


# ----------------------------------------------------------------------------- ranks
def max_over_ranks(value, world, device):
    """The largest of every rank's value (the job's time is its slowest rank's)."""
    if world <= 1:
        return float(value)
    import torch
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.MAX)
    return float(t.item())


# ----------------------------------------------------------------------------- serving
def serving_catalogue(W, seed=2106_06184 + 4):
    """The serving workload's models [(xyz, tri, mats, layered, a_max)] and, per model,
    its frequency bins."""
    from workloads.meshes import ellipsoid
    rng = np.random.default_rng(seed)
    models = []
    for i in range(W["n_models"] // 2):
        sub = int(rng.integers(1, 3))
        ax = rng.uniform(0.05, 0.2, 3) if i % 2 else np.full(3, rng.uniform(0.05, 0.2))
        eps = float(rng.uniform(2, 12))
        tand = float(rng.uniform(0, 0.02))
        a = float(ax.max())
        xyz, tri = ellipsoid(sub, tuple(ax), (0.0, 0.0, 1.2 * a))
        for layered in (False, True):
            models.append(dict(xyz=xyz, tri=tri, eps=eps, tand=tand, layered=layered, a=a))
    c0 = 299792458.0
    for m in models:
        ka = np.exp(np.linspace(np.log(0.1), np.log(2.0), W["n_freqs"]))
        m["freqs"] = [float(k * c0 / (2 * np.pi * m["a"])) for k in ka]
        # conductivity for the loss tangent at the middle of the band
        fm = m["freqs"][len(m["freqs"]) // 2]
        m["sigma"] = m["tand"] * 2 * np.pi * fm * 8.8541878128e-12 * m["eps"]
    return models


def serving_trace(W, step, nkeys):
    """Seeded request trace of one step: [(arrival_s, key, khat (n, 3), pol (n, 3))]."""
    rng = np.random.default_rng(2106_06184 + 1000 + step)
    perm = np.random.default_rng(2106_06184 + 999).permutation(nkeys)
    p = 1.0 / np.arange(1, nkeys + 1) ** W["zipf"]
    p /= p.sum()
    t = np.cumsum(rng.exponential(1.0 / W["rate"], W["requests"]))
    out = []
    for i in range(W["requests"]):
        key = int(perm[rng.choice(nkeys, p=p)])
        n = int(rng.integers(1, W["nrhs_max"] + 1))
        th = np.radians(rng.uniform(0, 70, n))
        ph = rng.uniform(-np.pi, np.pi, n)
        khat = np.stack([np.sin(th) * np.cos(ph), np.sin(th) * np.sin(ph), -np.cos(th)], axis=1)
        e_te = np.stack([-np.sin(ph), np.cos(ph), np.zeros(n)], axis=1)
        pol = np.where(rng.random((n, 1)) < 0.5, e_te, np.cross(e_te, khat))
        out.append((float(t[i] - t[0]), key, khat, pol))
    return out


def run_serving(args, rank, world):
    """Replays seeded Poisson request traces against the server in real time (a
    submitting thread sleeps until each arrival); a step is one trace.  value =
    right-hand sides solved per second from the first arrival to the last result;
    latency = submit -> result per request."""
    import threading
    import torch

    from paper_2106_06184_gb300 import sldm

    dev = int(os.environ.get("LOCAL_RANK", 0))
    torch.cuda.set_device(dev)
    W = WORKLOADS[args.workload]
    cat = serving_catalogue(W)
    free = sldm.Stack([(1.0, 1.0, 0.0, 0.0)])
    ground = sldm.Stack([(1.0, 1.0, 0.0, 0.0), (4.0, 1.0, 0.0, 0.05), (10.0, 1.0, 0.01, 0.0)], z_top=0.0)
    meshes = [sldm.Mesh(m["xyz"], m["tri"]) for m in cat]
    keys = [(mi, f) for mi, m in enumerate(cat) for f in m["freqs"]]

    def make_server(workers, max_batch, precision):
        srv = sldm.Server(workers=workers, max_batch=max_batch, precision=precision, budget_bytes=W["budget"])
        ids = [srv.add_model(meshes[i], ground if m["layered"] else free,
                             [(m["eps"], 1.0, m["sigma"], 0)]) for i, m in enumerate(cat)]
        return srv, ids

    def replay(srv, ids, step):
        trace = serving_trace(W, step, len(keys))
        xs = [np.zeros((len(kh), meshes[keys[k][0]].n_unknowns), complex) for _, k, kh, _ in trace]
        tickets = [None] * len(trace)

        def submit():
            t0 = time.perf_counter()
            for i, (ta, k, kh, po) in enumerate(trace):
                d = ta - (time.perf_counter() - t0)
                if d > 0:
                    time.sleep(d)
                mi, f = keys[k]
                tickets[i] = srv.submit(ids[mi], f, kh, po, xs[i], tol=W["tol"])

        t0 = time.perf_counter()
        th = threading.Thread(target=submit)
        th.start()
        th.join()
        res = [srv.wait(t, timeout=3600) for t in tickets]
        wall = time.perf_counter() - t0
        nrhs = sum(len(kh) for _, _, kh, _ in trace)
        lat = np.array([r["t_done"] - r["t_submit"] for r in res])
        bad = sum(r["code"] != sldm.OK for r in res)
        h2d = sum(kh.nbytes * 2 for _, _, kh, _ in trace)
        d2h = sum(x.nbytes for x in xs)
        return dict(wall=wall, nrhs=nrhs, lat=lat, bad=bad, hits=sum(r["cache_hit"] for r in res),
                    relres=max(r["relres"] for r in res), h2d=h2d, d2h=d2h, xs=xs)

    srv, ids = make_server(W["workers"], W["max_batch"], W["precision"])
    for i in range(args.warmup):
        replay(srv, ids, i)
    clocks = ClockSampler(dev)
    clocks.start()
    sldm.timers_reset()
    sldm.timers_enable(True)
    launches0 = sldm.launch_count()
    runs = [replay(srv, ids, args.warmup + i) for i in range(args.steps)]
    launches = sldm.launch_count() - launches0
    sldm.timers_enable(False)
    timers = sldm.timers_read()
    clk = clocks.stop()
    st = srv.stats()
    srv.close()
    wall = sum(r["wall"] for r in runs)
    nrhs = sum(r["nrhs"] for r in runs)
    lat = np.concatenate([r["lat"] for r in runs])
    value = nrhs / wall
    # the plain FP64 single-solve path on the first timed step's trace (cold cache, then warm)
    base, bids = make_server(1, 1, 0)
    replay(base, bids, args.warmup)
    b = replay(base, bids, args.warmup)
    base.close()
    # the two paths' currents on that trace agree to the solve tolerance times the conditioning
    agree = max(np.linalg.norm(x - y) / max(np.linalg.norm(y), 1e-300) for x, y in zip(runs[0]["xs"], b["xs"]))
    kernel_ms = {k: round(v[0] / args.steps, 4) for k, v in sorted(timers.items(), key=lambda kv: -kv[1][0])}
    out = {
        "metric": METRIC, "value": value, "unit": "solves/s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": wall / args.steps * 1e3, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "c64+c64 (FP64-accurate residual)", "data": "synthetic",
        "config": {"workload": args.workload, "requests_per_step": W["requests"], "arrival_rate_per_s": W["rate"],
                   "keys": len(keys), "workers": W["workers"], "max_batch": W["max_batch"],
                   "budget_bytes": W["budget"], "l2": "the trace's operators exceed L2 in aggregate; no flush"},
        "latency_ms": {"p50": float(np.percentile(lat, 50) * 1e3), "p99": float(np.percentile(lat, 99) * 1e3),
                       "max": float(lat.max() * 1e3)},
        "server": {k: st[k] for k in ("requests", "rhs", "batches", "hits", "misses", "evictions", "rejected",
                                      "cached_ops", "cached_bytes")},
        "failed_requests": int(sum(r["bad"] for r in runs)),
        "relres_max": float(max(r["relres"] for r in runs)),
        "fp64_single_baseline": {"value": b["nrhs"] / b["wall"], "unit": "solves/s",
                                 "latency_ms": {"p50": float(np.percentile(b["lat"], 50) * 1e3),
                                                "p99": float(np.percentile(b["lat"], 99) * 1e3)},
                                 "failed_requests": int(b["bad"]), "workers": 1, "max_batch": 1, "precision": "f64",
                                 "trace": "the first timed step's, warm cache"},
        "served_vs_fp64_single_max_rel_diff": float(agree),
        "e2e": {"value": value, "unit": "solves/s", "h2d_bytes_per_step": int(runs[0]["h2d"]),
                "d2h_bytes_per_step": int(runs[0]["d2h"]),
                "note": "requests carry host arrays (plane waves in, currents out): the served value is end to end"},
        "gpu_launches": int(launches), "clocks": clk, "kernel_ms_per_step": kernel_ms,
    }
    return out


# ----------------------------------------------------------------------------- sweep
def sweep_catalogue(W, seed=2106_06184 + 3):
    """The sweep's instances [dict(xyz, tri, eps, sigma, freqs)] and the incidence set."""
    from workloads.meshes import ellipsoid
    rng = np.random.default_rng(seed)
    out = []
    c0 = 299792458.0
    for i in range(W["n_inst"]):
        if i == W["n_inst"] - 1:  # the large instance: a sub-4 sphere
            ax, sub, eps, tand = np.full(3, 0.1), 4, 4.0, 0.0
        else:
            sub = int(rng.integers(2, 4))
            ax = rng.uniform(0.05, 0.2, 3) if i % 2 else np.full(3, rng.uniform(0.05, 0.2))
            eps, tand = float(rng.uniform(2, 12)), float(rng.uniform(0, 0.02))
        xyz, tri = ellipsoid(sub, tuple(ax), (0.0, 0.0, 0.0))
        a, h = float(ax.max()), float(np.mean(ax))
        f_lo = 0.01 * c0 / (2 * np.pi * a)
        f_hi = c0 / (10 * np.sqrt(eps) * h)
        freqs = [float(f) for f in np.exp(np.linspace(np.log(f_lo), np.log(f_hi), W["n_freqs"]))]
        fm = freqs[len(freqs) // 2]
        sigma = tand * 2 * np.pi * fm * 8.8541878128e-12 * eps
        out.append(dict(xyz=xyz, tri=tri, eps=eps, sigma=sigma, freqs=freqs))
    th = np.radians((np.arange(W["n_angles_inc"]) + 0.5) * 22.5)
    khat = np.stack([np.sin(th), np.zeros_like(th), -np.cos(th)], axis=1)
    pol = np.stack([np.cos(th), np.zeros_like(th), np.sin(th)], axis=1)  # theta-polarised (in the xz plane)
    return out, khat, pol


def _register_sweep_instances():
    """One plain workload per sweep instance (its middle frequency, the sweep's
    plane waves), for the oracle's sampled timing of a request of that instance."""
    for name, W in list(WORKLOADS.items()):
        if W.get("kind") != "sweep":
            continue
        cat, khat, pol = sweep_catalogue(W)
        for i, c in enumerate(cat):
            WORKLOADS[f"{name}-inst{i}"] = dict(
                mesh=(lambda c=c: (c["xyz"], c["tri"])), obj=None, mats=[(c["eps"], 1.0, c["sigma"])],
                bg=(1.0, 1.0, 0.0, 0.0), freq=c["freqs"][len(c["freqs"]) // 2], precision=W["precision"], tol=W["tol"],
                khat=khat.tolist(), pol=pol.tolist(), n_angles=0)


_register_sweep_instances()


def run_sweep(args, rank, world):
    """The whole sweep as one step: every (instance, frequency) request submitted at
    once to the serving loop with an emptied cache (so every step assembles all
    operators); value = plane waves solved per second of the step."""
    import torch

    from paper_2106_06184_gb300 import sldm

    dev = int(os.environ.get("LOCAL_RANK", 0))
    torch.cuda.set_device(dev)
    W = WORKLOADS[args.workload]
    cat, khat, pol = sweep_catalogue(W)
    free = sldm.Stack([(1.0, 1.0, 0.0, 0.0)])
    meshes = [sldm.Mesh(c["xyz"], c["tri"]) for c in cat]

    def one_sweep(srv, ids):
        xs, tickets = [], []
        t0 = time.perf_counter()
        for i, c in enumerate(cat):
            for f in c["freqs"]:
                x = np.zeros((len(khat), meshes[i].n_unknowns), complex)
                xs.append(x)
                tickets.append(srv.submit(ids[i], f, khat, pol, x, tol=W["tol"]))
        res = [srv.wait(t, timeout=3600) for t in tickets]
        wall = time.perf_counter() - t0
        srv.flush()
        return wall, res, xs

    def make(workers):
        srv = sldm.Server(workers=workers, max_batch=W["max_batch"], precision=W["precision"], budget_bytes=W["budget"])
        ids = [srv.add_model(meshes[i], free, [(c["eps"], 1.0, c["sigma"], 0)]) for i, c in enumerate(cat)]
        return srv, ids

    srv, ids = make(W["workers"])
    for _ in range(args.warmup):
        one_sweep(srv, ids)
    clocks = ClockSampler(dev)
    clocks.start()
    sldm.timers_reset()
    sldm.timers_enable(True)
    launches0 = sldm.launch_count()
    runs = [one_sweep(srv, ids) for _ in range(args.steps)]
    launches = sldm.launch_count() - launches0
    sldm.timers_enable(False)
    timers = sldm.timers_read()
    clk = clocks.stop()
    st = srv.stats()
    srv.close()
    nrhs = len(khat) * sum(len(c["freqs"]) for c in cat)
    wall = sum(r[0] for r in runs)
    value = nrhs * args.steps / wall
    lat = np.array([r_["t_done"] - r_["t_submit"] for r in runs for r_ in r[1]])
    bad = sum(r_["code"] != sldm.OK for r in runs for r_ in r[1])
    relres = max(r_["relres"] for r in runs for r_ in r[1])
    # one worker, same sweep
    s1, ids1 = make(1)
    one_sweep(s1, ids1)
    w1, res1, xs1 = one_sweep(s1, ids1)
    s1.close()
    agree = max(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300) for a, b in zip(runs[0][2], xs1))
    # the crossover the autotuner picked, per instance at the middle frequency
    tc_from = []
    for i, c in enumerate(cat):
        op = sldm.Operator(meshes[i], free, [(c["eps"], 1.0, c["sigma"], 0)], c["freqs"][len(c["freqs"]) // 2],
                           precision=W["precision"])
        tc_from.append(int(op.tc_from))
        del op
    kernel_ms = {k: round(v[0] / args.steps, 4) for k, v in sorted(timers.items(), key=lambda kv: -kv[1][0])}
    return {
        "metric": METRIC, "value": value, "unit": "solves/s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": wall / args.steps * 1e3, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "c64 (FP64 singular terms)", "data": "synthetic",
        "config": {"workload": args.workload, "instances": len(cat),
                   "triangles": [int(len(c["tri"])) for c in cat], "freqs_per_instance": W["n_freqs"],
                   "plane_waves_per_freq": len(khat), "workers": W["workers"], "max_batch": W["max_batch"],
                   "l2": "each step assembles every operator (cache emptied); no flush"},
        "latency_ms": {"p50": float(np.percentile(lat, 50) * 1e3), "p99": float(np.percentile(lat, 99) * 1e3)},
        "failed_requests": int(bad), "relres_max": float(relres),
        "one_worker": {"value": nrhs / w1, "unit": "solves/s", "ms_per_step": w1 * 1e3,
                       "max_rel_diff_vs_two_workers": float(agree)},
        "autotune_tc_from": tc_from,
        "server": {k: st[k] for k in ("requests", "rhs", "batches", "hits", "misses")},
        "e2e": {"value": value, "unit": "solves/s", "h2d_bytes_per_step": int(2 * khat.nbytes * len(runs[0][1])),
                "d2h_bytes_per_step": int(sum(x.nbytes for x in runs[0][2])),
                "note": "requests carry host arrays: the value is end to end"},
        "gpu_launches": int(launches), "clocks": clk, "kernel_ms_per_step": kernel_ms,
    }


# ----------------------------------------------------------------------------- our arm
def run_ours(args, rank, world):
    import torch

    from paper_2106_06184_gb300 import sldm

    dev = int(os.environ.get("LOCAL_RANK", 0))
    torch.cuda.set_device(dev)
    W = WORKLOADS[args.workload]
    xyz, tri = W["mesh"]()
    obj_ids = _obj_ids(W)
    mesh = sldm.Mesh(xyz, tri, obj_ids)
    stack = _stack(sldm, W)
    freqs = _freqs(W)
    theta = np.radians(np.linspace(0.0, W.get("rcs_theta_max_deg", 180.0), W["n_angles"]))
    phi = np.zeros_like(theta)
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device="cuda")

    nrhs = _nrhs(W)
    ports = (sldm.Ports([sldm.port_ring(mesh, o, sv, c) for o, sv, c in W["ports"]]) if "ports" in W else None)
    s_params = {}

    def excite(op, b):
        if ports is not None:
            op.port_rhs(ports, np.eye(nrhs), b)   # one port driven per column, the others shorted
        else:
            op.rhs_planewave(W["khat"], W["pol"], b)

    def post(op, x, i):
        """RCS of every plane wave, or the ports' S matrix (recorded per frequency)."""
        if ports is not None:
            Y = op.port_currents(x, ports, ncols=nrhs)
            Sm = sldm.sparams(Y, W["z0"])
            s_params[freqs[i % len(freqs)]] = Sm
            return Sm
        return op.farfield_n(x, theta, phi, nrhs) if W["n_angles"] else None

    def step_device(i):
        op = sldm.Operator(mesh, stack, W["mats"], freqs[i % len(freqs)], precision=W["precision"])
        b = torch.zeros((nrhs, op.N), dtype=torch.complex128, device="cuda")
        excite(op, b)
        x = torch.zeros_like(b)
        info = op.solve(b, x, nrhs=nrhs, tol=W["tol"], maxit=W.get("maxit", 2000), check=False)
        return op, info, post(op, x, i)

    for i in range(args.warmup):
        op, info, rcs = step_device(i)
        del op
    torch.cuda.synchronize()
    if world > 1:
        torch.distributed.barrier()
    clocks = ClockSampler(dev)
    clocks.start()
    sldm.timers_reset()
    sldm.timers_enable(True)
    times, iters, relres = [], [], []
    launches0 = sldm.launch_count()
    t_wall0 = time.perf_counter()
    for i in range(args.steps):
        flush.zero_()
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        op, info, rcs = step_device(i)
        e1.record()
        torch.cuda.synchronize()
        times.append(e0.elapsed_time(e1))
        iters.append(info["iters"])
        relres.append(info["relres"])
        del op
    t_wall = time.perf_counter() - t_wall0
    launches = sldm.launch_count() - launches0
    sldm.timers_enable(False)
    timers = sldm.timers_read()
    units = {k: sldm.timer_units(k) for k in timers}
    clk = clocks.stop()
    torch.cuda.synchronize()
    if world > 1:
        torch.distributed.barrier()
    total_ms = max_over_ranks(float(sum(times)), world, "cuda")

    # ---- e2e: the same step through the public API with host buffers
    e2e_times = []
    h2d = d2h = 0
    n_e2e = 0 if args.no_e2e else max(3, min(args.steps, W.get("e2e_steps", 10)))
    for i in range(n_e2e):
        fi = (i * len(freqs)) // n_e2e + len(freqs) // (2 * n_e2e)  # spread over the sweep
        flush.zero_()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        m2 = sldm.Mesh(xyz, tri, obj_ids)                       # H2D: vertices and triangles
        op2 = sldm.Operator(m2, stack, W["mats"], freqs[fi % len(freqs)], precision=W["precision"])
        bh = np.zeros((nrhs, op2.N), complex)
        excite(op2, bh)                                         # D2H: b
        xh = np.zeros((nrhs, op2.N), complex)
        op2.solve(bh, xh, nrhs=nrhs, tol=W["tol"], maxit=W.get("maxit", 2000), check=False)  # H2D: b, D2H: x
        rcs2 = post(op2, xh, fi)                                # H2D: x; D2H: rcs or port currents
        rcs2 = np.zeros(0) if rcs2 is None else np.asarray(rcs2)
        e2e_times.append(time.perf_counter() - t0)
        if i == 0:
            h2d = (xyz.nbytes + tri.astype(np.int32).nbytes + bh.nbytes + xh.nbytes
                   + (nrhs * (theta.nbytes + phi.nbytes) if W["n_angles"] else 0)
                   + (0 if obj_ids is None else np.asarray(obj_ids, np.int32).nbytes))
            d2h = bh.nbytes + xh.nbytes + rcs2.nbytes
        del op2, m2
    n_units = args.steps * world * nrhs
    value = n_units / (total_ms / 1e3)
    e2e_value = world * nrhs / statistics.median(e2e_times) if e2e_times else None

    # ---- rooflines (live CUDA-event timings; algorithmic units counted by the library)
    hbm, hbm_src = peaks()
    ne, nt, nobj = mesh.ne, mesh.nt, mesh.nobj
    uv, tp, tm = mesh.edges()
    tri_obj = np.zeros(nt, np.int64) if obj_ids is None else np.asarray(obj_ids)
    obj_sizes = [(int(np.sum(tri_obj[tp] == o)), int(np.sum(tri_obj == o))) for o in range(nobj)]
    fp64_fill = W["precision"] in (0, 2)   # c64x2 fills in FP64, then splits

    def matvec_entry(name):
        """HBM roofline of one GEMV stage: matrix bytes per launch / mean launch time."""
        if name not in timers or units.get(name, 0) <= 0:
            return None
        ms, cnt = timers[name]
        per_launch = units[name] / cnt
        achieved = per_launch / (ms / cnt / 1e3) / 1e9
        e = {"kernel": name, "bound": "hbm", "achieved": achieved, "peak": hbm, "unit": "GB/s", "frac": achieved / hbm,
             "peak_source": hbm_src, "traffic": None, "algorithmic_unit": per_launch, "launches": cnt,
             "ms_per_launch": ms / cnt}
        kern = "gemm_tc_kernel" if "gemm_tc" in timers else ("gemv_tile_kernel" if nrhs > 1 else "gemv_jobs_kernel")
        tr = GEMV_TRAFFIC.get(kern)
        if name == "gemv_main" and tr and kernel_sha(kern, tr["file"]) == tr["sha"]:
            e["traffic"] = tr["per_alg_byte"] * per_launch
            e["traffic_source"] = "ncu capture of the 4x4 case (same kernel source), scaled by algorithmic bytes"
        e["kernel_impl"] = kern
        return e

    def fill_entry(name):
        """ALU roofline of a bulk fill kernel: Green's-function evaluations per second."""
        if name not in timers or units.get(name, 0) <= 0:
            return None
        ms, cnt = timers[name]
        per_launch = units[name] / cnt
        evals = per_launch / (ms / cnt / 1e3)
        if name == "fill_reflected_bulk":  # FP64 whatever the operator's precision
            peak = FP64_OPS_PER_S / FP64_OPS_PER_EVAL_REFL
            return {"kernel": name, "bound": "alu", "achieved": evals / 1e9, "peak": peak / 1e9, "unit": "Geval/s",
                    "frac": evals / peak, "peak_source": "derived (FP64 pipe)", "traffic": None,
                    "algorithmic_unit": per_launch, "launches": cnt, "ms_per_launch": ms / cnt, "precision": "fp64",
                    "fp64_ops_per_eval": FP64_OPS_PER_EVAL_REFL}
        peak = FILL_F64_PEAK_EVALS if fp64_fill else FILL_F32_PEAK_EVALS
        return {"kernel": name, "bound": "alu", "achieved": evals / 1e9, "peak": peak / 1e9, "unit": "Geval/s",
                "frac": evals / peak, "peak_source": "derived (FP64 pipe)" if fp64_fill else "derived (SFU)",
                "traffic": None, "algorithmic_unit": per_launch, "launches": cnt, "ms_per_launch": ms / cnt,
                "precision": "fp64" if fp64_fill else "fp32"}

    roof_mv = matvec_entry("gemv_main")
    roof_gs = None
    if "gram_schmidt" in timers and units.get("gram_schmidt", 0) > 0:
        # classical Gram-Schmidt twice: two dot and two update passes over the basis
        ms, cnt = timers["gram_schmidt"]
        ach = units["gram_schmidt"] / (ms / 1e3) / 1e9
        roof_gs = {"kernel": "gram_schmidt", "bound": "hbm", "achieved": ach, "peak": hbm, "unit": "GB/s",
                   "frac": ach / hbm, "peak_source": hbm_src, "traffic": None,
                   "algorithmic_unit": units["gram_schmidt"] / cnt, "launches": 4 * cnt, "ms_per_launch": ms / cnt / 4}
    fills = [f for f in (fill_entry(k) for k in ("fill_L_bulk", "fill_K_bulk", "fill_reflected_bulk")) if f]
    roof_fill = max(fills, key=lambda f: f["ms_per_launch"] * f["launches"]) if fills else None
    # the direct solves: the batched look-ahead LU (small objects) and the blocked LU (large ones)
    # (the FP32 approximate inverses of inner-solve objects run inside "nested_inverse": not FP64 work)
    lu_ms = sum(timers[k][0] for k in ("lu_coop", "lu_blocked") if k in timers) - timers.get("nested_inverse", (0.0, 0))[0]
    roof_lu = None
    if lu_ms > 0 and W["precision"] in (0, 2):
        ms = lu_ms / args.steps
        fl = lu_flops(obj_sizes, W["precision"])
        ach = fl / (ms / 1e3) / 1e12
        roof_lu = {"kernel": "lu", "bound": "alu", "achieved": ach, "peak": FP64_PEAK_TFLOPS, "unit": "TFLOP/s",
                   "frac": ach / FP64_PEAK_TFLOPS, "peak_source": "derived (FP64 pipe)", "traffic": None,
                   "algorithmic_unit": fl, "launches": None, "ms_per_launch": None}
        timers["lu"] = (lu_ms, sum(timers[k][1] for k in ("lu_coop", "lu_blocked") if k in timers))
    # the dominant kernel of the step among these
    cands = [(roof_mv, "gemv_main"), (roof_fill, roof_fill["kernel"] if roof_fill else None), (roof_lu, "lu")]
    cands = [(r, k) for r, k in cands if r is not None]
    roof = None
    if cands:
        r, k = max(cands, key=lambda rk: timers[rk[1]][0])
        roof = dict(r)
        roof["share_of_step"] = timers[k][0] / total_ms if world == 1 else None
    kernel_ms = {k: round(v[0] / args.steps, 4) for k, v in sorted(timers.items(), key=lambda kv: -kv[1][0])}
    out = {
        "metric": METRIC,
        "value": value, "unit": "solves/s", "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": total_ms / args.steps, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": {0: "c128", 1: "c64", 2: "c64x2"}[W["precision"]], "data": "synthetic",
        "config": {"workload": args.workload, "n_triangles": nt, "n_edges": ne, "n_objects": nobj,
                   "n_unknowns": mesh.n_unknowns,
                   "freq_hz": freqs if len(freqs) > 1 else freqs[0], "rel_residual": W["tol"],
                   "rhs_per_step": nrhs,
                   "rcs_angles": W["n_angles"], "background": "layered" if "layers" in W else "homogeneous",
                   "parallelism": f"replicas x{world}", "l2": "flushed between steps (512 MB write)"},
        "latency_ms": {"p50": float(np.percentile(times, 50)), "p99": float(np.percentile(times, 99))},
        "gmres": {"iters": int(np.median(iters)), "relres_max": float(max(relres))},
        "roofline": roof, "roofline_matvec": roof_mv, "roofline_fill": roof_fill, "roofline_gram_schmidt": roof_gs,
        "kernel_ms_per_step": kernel_ms,
        "gpu_launches": int(launches),
        "clocks": clk,
        "e2e": {"value": e2e_value, "unit": "solves/s", "h2d_bytes_per_step": int(h2d), "d2h_bytes_per_step": int(d2h),
                "latency_ms_p50": 1e3 * statistics.median(e2e_times) if e2e_times else None},
        "wall_s_timed": t_wall,
    }
    if ports is not None:
        out["ports"] = {"n": nrhs, "z0_ohm": W["z0"], "ring_edges": [int(ports.ptr[p + 1] - ports.ptr[p])
                                                                    for p in range(nrhs)],
                        "s11": {f"{f / 1e6:.2f} MHz": [float(abs(Sm[0, 0])), float(np.degrees(np.angle(Sm[0, 0])))]
                                for f, Sm in sorted(s_params.items())},
                        "s11_format": "[|S11|, phase deg]"}
        out["config"]["ports"] = nrhs
    return out


METRIC = ("solves/s (per plane-wave right-hand side: assemble + RHS + GMRES to the stated relative residual; "
          "+ bistatic RCS where the workload asks for it; a port workload counts one right-hand side per port "
          "and adds the port currents and S matrix)")


# ----------------------------------------------------------------------------- oracle timing
# The oracle as it stands, single-threaded on the host.  The small sphere is
# solved whole; larger workloads are timed on a bounded sample and extrapolated:
# uniformly drawn triangle pairs of every fill (scaled by the pair counts), the
# reflected fill on a random subset of triangles (scaled by the square of the
# fraction), the layered tables whole, and the dense solves (Y of each object by
# LU of M_l, the final system by LU) on random matrices 1/d of the size, d at
# least 2 and large enough for an order of at most 2,048 (scaled by d^3).
ORACLE_FULL = r"""
import sys, time, numpy as np
sys.path.insert(0, {root!r})
from workloads.meshes import icosphere
from oracle.topology import Mesh
from oracle import system as S, farfield
xyz, tri = icosphere(2, 0.1)
t0 = time.perf_counter()
m = Mesh(xyz, tri)
A = S.assemble(m, [S.Material(4.0, 1.0, 0.0)], S.Material(1.0, 1.0, 0.0), 300e6)
x = S.solve(A, S.rhs(A))
th = np.radians(np.linspace(0, 180, 181))
rcs = farfield.rcs(m, A.k0, S.j_delta(A, x), th)
print(time.perf_counter() - t0)
"""

ORACLE_SAMPLED = r"""
import sys, time, numpy as np
sys.path.insert(0, {root!r})
import scipy.linalg as sla
import bench
from oracle.topology import Mesh
from oracle import system as S, fill as F, layered as LY
W = bench.WORKLOADS[{name!r}]
freq = bench._freqs(W)[{step} % len(bench._freqs(W))]
xyz, tri = W["mesh"]()
obj = bench._obj_ids(W)
rng = np.random.default_rng(2106_06184)
t_all = time.perf_counter()
m = Mesh(xyz, tri, obj)
omega = 2 * np.pi * freq
k0 = omega / S.C0
if "layers" in W:
    st = LY.Stack([(l[0], l[1], l[2], l[3] if l[3] > 0 else np.inf) for l in W["layers"]], z_top=W["z_top"],
                  bottom=W["bottom"])
    lay = W["mats"][0][3]
    bg = S.Material(*st.layers[lay][:3])
else:
    st = None
    bg = S.Material(*W["bg"][:3])
kb = S.wavenumber(bg, k0)
P = m.xyz[m.tri]
Pb = m.bxyz[m.btri]
est = 0.0
NS = {npairs}
DMAX = 2048  # largest order of a timed dense solve

def timed_pairs(fn, k, ta, tb, Psrc, touch_fn, total, nsrc):
    # uniformly drawn pairs; with split sources: the far-pair rule, then grouped by the size
    # of the source's quadrature.  The quadrature rules of the drawn sources are timed apart
    # and scaled to the fill's nsrc sources (the fill builds each source's rule once).
    t_rules = 0.0
    t0 = time.perf_counter()
    if not F.needs_split(k, Psrc).any():
        for c in range(0, len(ta), F.CHUNK):
            fn(m, k, ta[c:c + F.CHUNK], tb[c:c + F.CHUNK])
    else:
        keep = F._kept(k, P[ta], Psrc[tb], touch_fn(ta, tb))
        a, b = ta[keep], tb[keep]
        t1 = time.perf_counter()
        rules = {{int(s): F.source_rule(Psrc[s], k) for s in np.unique(b)}}
        t_rules = (time.perf_counter() - t1)
        t_rules_est = t_rules * nsrc / max(len(rules), 1)
        ns = np.array([len(rules[int(s)][1]) for s in b], dtype=np.int64)
        for n in np.unique(ns):
            sel = np.nonzero(ns == n)[0]
            step = max(1, F.CHUNK * 6 // int(n))
            for c in range(0, len(sel), step):
                idx = sel[c:c + step]
                pts = np.stack([rules[int(b[i])][0] for i in idx])
                w = np.stack([rules[int(b[i])][1] for i in idx])
                fn(m, k, a[idx], b[idx], (pts, w))
        return (time.perf_counter() - t0 - t_rules) * total / len(ta) + t_rules_est
    return (time.perf_counter() - t0) * total / len(ta)

touch_L = lambda a, b: F._touch_primal(m.tri, a, b)
touch_K = lambda a, b: F._touch_bary(m, a, b) > 0
# global L with the background's k (the equivalent blocks are its diagonal blocks)
ta = rng.integers(0, m.nt, NS); tb = rng.integers(0, m.nt, NS)
est += timed_pairs(F._L_pairs, kb, ta, tb, P, touch_L, float(m.nt) ** 2, m.nt)
for o in range(m.nobj):
    t0_, t1_ = m.tri_range[o]
    mat = S.Material(*W["mats"][o][:3])
    ko = S.wavenumber(mat, k0)
    n_o = t1_ - t0_
    ns = max(NS // m.nobj, 64)
    ta = rng.integers(t0_, t1_, ns); tb = rng.integers(t0_, t1_, ns)
    est += timed_pairs(F._L_pairs, ko, ta, tb, P, touch_L, float(n_o) ** 2, n_o)
    for k in (ko, kb):
        ta = rng.integers(t0_, t1_, ns); cb = rng.integers(6 * t0_, 6 * t1_, ns)
        est += timed_pairs(F._K_pairs, k, ta, cb, Pb, touch_K, 6.0 * n_o ** 2, 6 * n_o)
    # Y = M_l^-1 R_l on random matrices 1/d of the size (order at most DMAX), scaled by d^3
    e0_, e1_ = m.edge_range[o]
    d = max({ddiv}, -(-(e1_ - e0_ + n_o - 1) // DMAX))
    n, r = (e1_ - e0_ + n_o - 1) // d, (e1_ - e0_) // d
    A_ = rng.standard_normal((n, n)) + 1j * rng.standard_normal((n, n))
    B_ = rng.standard_normal((n, r)) + 1j * rng.standard_normal((n, r))
    t0 = time.perf_counter(); np.linalg.solve(A_, B_); est += d ** 3 * (time.perf_counter() - t0)
if st is not None:
    # the tables of default_tables, timed at 16 and 32 of their 256 rho rows (every
    # z + z' and |z - z'| column, every Sommerfeld node): the cost is affine in the
    # rows (Bessel functions and the node sum per row), so the 256-row build is
    # extrapolated linearly
    lo, hi = m.xyz.min(axis=0), m.xyz.max(axis=0)
    span = np.linalg.norm(hi - lo) * 1.01
    edge = np.min(np.linalg.norm(m.xyz[m.E.uv[:, 0]] - m.xyz[m.E.uv[:, 1]], axis=1))
    TABLE_S = {table_s}
    if TABLE_S is None:
        tt = []
        for nr in (16, 32):
            t0 = time.perf_counter()
            T = LY.build_tables(st, lay, omega, 1e-3 * edge, span, lo[2], hi[2], nr=nr)
            tt.append(time.perf_counter() - t0)
        TABLE_S = tt[0] + (tt[1] - tt[0]) * (256 - 16) / 16
    else:
        # the same tables as an earlier sample of this run (same stack, frequency and
        # extent): their measured time is reused; a coarse table serves the fill below
        T = LY.build_tables(st, lay, omega, 1e-3 * edge, span, lo[2], hi[2], nr=16, ns=16, nd=16)
    est += TABLE_S
    sub = np.sort(rng.choice(m.nt, size=min(m.nt, {nsub}), replace=False))
    t0 = time.perf_counter()
    LY.fill_reflected(m, st, lay, omega, T, sub)
    est += (time.perf_counter() - t0) * (m.nt / len(sub)) ** 2
N = 2 * m.ne + m.nt - m.nobj
d = max({ddiv}, -(-N // DMAX))
A_ = rng.standard_normal((N // d, N // d)) + 1j * rng.standard_normal((N // d, N // d))
t0 = time.perf_counter(); sla.lu_solve(sla.lu_factor(A_), np.ones(N // d)); est += (N / (N // d)) ** 3 * (time.perf_counter() - t0)
print(est, time.perf_counter() - t_all, TABLE_S if st is not None else -1.0)
"""

_TABLE_S = {}  # (workload, frequency index) -> seconds of the oracle's layered tables, measured once per run


def oracle_step_seconds(name=None, step=0, quick=False):
    """One oracle solve of the workload on one host thread: (seconds per step, sample
    description, extrapolated?, seconds actually spent).  quick: a smaller sample
    (the reference arm times one per step)."""
    name = name or DEFAULT_WORKLOAD
    env = dict(os.environ, OMP_NUM_THREADS="1", OPENBLAS_NUM_THREADS="1", MKL_NUM_THREADS="1")
    if name.startswith("sphere"):
        script = ORACLE_FULL.format(root=ROOT)
        sample = "one full solve of the workload (oracle assemble + dense LU + RCS), single thread"
        extrap = False
    else:
        npairs, nsub, ddiv = (1000, 48, 4) if quick else (3000, 96, 2)
        W = WORKLOADS[name]
        key = (name, step % len(_freqs(W)))
        script = ORACLE_SAMPLED.format(root=ROOT, name=name, step=step, npairs=npairs, nsub=nsub, ddiv=ddiv,
                                       table_s=repr(_TABLE_S.get(key)))
        sample = (f"extrapolated from a sample at frequency index {step}: {npairs} uniformly drawn triangle pairs per "
                  f"fill (global L, each object's L, Kbar with k and k_l), the reflected fill on {nsub} random "
                  f"triangles, the layered tables at 16 and 32 of 256 rho rows (extrapolated linearly; measured once per "
                  f"run and frequency), the dense solves on matrices 1/d of the size (d >= {ddiv}, "
                  "order <= 2048, scaled by d^3); "
                  "single thread")
        extrap = True
    r = subprocess.run([sys.executable, "-c", script], capture_output=True, text=True, env=env, timeout=300, cwd=ROOT)
    if r.returncode != 0:
        raise RuntimeError(r.stderr[-2000:])
    vals = [float(v) for v in r.stdout.strip().splitlines()[-1].split()]
    if len(vals) > 2 and vals[2] >= 0 and not name.startswith("sphere"):
        _TABLE_S.setdefault(key, vals[2])
    return vals[0], sample, extrap, (vals[1] if len(vals) > 1 else vals[0])


def oracle_all_cores(name, step, ncores):
    """The oracle on every host core: ncores single-threaded copies of the same
    sampled solve run at once (independent requests, as the GPU's replicas), each
    extrapolated as above; aggregate solves/s = sum of the copies' rates.
    Returns (aggregate steps/s, wall seconds spent)."""
    name = name or DEFAULT_WORKLOAD
    env = dict(os.environ, OMP_NUM_THREADS="1", OPENBLAS_NUM_THREADS="1", MKL_NUM_THREADS="1")
    if name.startswith("sphere"):
        script = ORACLE_FULL.format(root=ROOT)
    else:
        key = (name, step % len(_freqs(WORKLOADS[name])))
        script = ORACLE_SAMPLED.format(root=ROOT, name=name, step=step, npairs=1000, nsub=48, ddiv=4,
                                       table_s=repr(_TABLE_S.get(key)))
    t0 = time.perf_counter()
    procs = [subprocess.Popen([sys.executable, "-c", script], stdout=subprocess.PIPE, stderr=subprocess.PIPE, text=True,
                              env=env, cwd=ROOT) for _ in range(ncores)]
    rate = 0.0
    for pr in procs:
        out, err = pr.communicate(timeout=600)
        if pr.returncode != 0:
            raise RuntimeError(err[-2000:])
        rate += 1.0 / float(out.strip().splitlines()[-1].split()[0])
    return rate, time.perf_counter() - t0


def cpu_model():
    try:
        for line in open("/proc/cpuinfo"):
            if line.lower().startswith(("model name", "cpu part")):
                return line.split(":", 1)[1].strip()
    except Exception:
        pass
    return platform.processor() or platform.machine()


ORACLE_SERVING = r"""
import sys, time, numpy as np
sys.path.insert(0, {root!r})
import scipy.linalg as sla
import bench
from oracle.topology import Mesh
from oracle import system as S, layered as LY
W = bench.WORKLOADS[{name!r}]
cat = bench.serving_catalogue(W)
keys = [(mi, f) for mi, m in enumerate(cat) for f in m["freqs"]]
ground = LY.Stack([(1.0, 1.0, 0.0, np.inf), (4.0, 1.0, 0.0, 0.05), (10.0, 1.0, 0.01, np.inf)], z_top=0.0)
trace = bench.serving_trace(W, {step}, len(keys))
t_all = time.perf_counter()
nrhs = 0
for ta, k, kh, po in trace:
    mi, f = keys[k]
    m = cat[mi]
    mesh = Mesh(m["xyz"], m["tri"])
    mat = S.Material(m["eps"], 1.0, m["sigma"])
    if m["layered"]:
        A = S.assemble(mesh, [mat], ground, f, layer=0)
    else:
        A = S.assemble(mesh, [mat], S.Material(), f)
    lu = sla.lu_factor(A.Z)
    for r in range(len(kh)):
        sla.lu_solve(lu, S.rhs(A, khat=kh[r], pol=po[r]))
    nrhs += len(kh)
    if time.perf_counter() - t_all > {budget_s}:
        break
print(time.perf_counter() - t_all, nrhs)
"""


ORACLE_SWEEP = r"""
import sys, time, numpy as np
sys.path.insert(0, {root!r})
import scipy.linalg as sla
import bench
from oracle.topology import Mesh
from oracle import system as S
W = bench.WORKLOADS[{name!r}]
cat, khat, pol = bench.sweep_catalogue(W)
t_all = time.perf_counter()
nrhs = 0
# the sub-4 sphere (dense order 20,479) takes the oracle far beyond a bounded sample:
# it is left out, which favours the oracle
order = [(i, f) for i, c in enumerate(cat) if len(c["tri"]) <= 1280 for f in c["freqs"]]
rng = np.random.default_rng({step})
for j in rng.permutation(len(order)):
    i, f = order[j]
    c = cat[i]
    A = S.assemble(Mesh(c["xyz"], c["tri"]), [S.Material(c["eps"], 1.0, c["sigma"])], S.Material(), f)
    lu = sla.lu_factor(A.Z)
    for r in range(len(khat)):
        sla.lu_solve(lu, S.rhs(A, khat=khat[r], pol=pol[r]))
    nrhs += len(khat)
    if time.perf_counter() - t_all > {budget_s}:
        break
print(time.perf_counter() - t_all, nrhs)
"""


def oracle_serving(name, step, budget_s=20.0):
    """The oracle on the serving trace of `step`, request by request (assembly of the
    dense system, LU, one back substitution per plane wave; no cache), in order
    until budget_s seconds are spent: (seconds, right-hand sides solved)."""
    env = dict(os.environ, OMP_NUM_THREADS="1", OPENBLAS_NUM_THREADS="1", MKL_NUM_THREADS="1")
    tmpl = ORACLE_SWEEP if WORKLOADS[name].get("kind") == "sweep" else ORACLE_SERVING
    script = tmpl.format(root=ROOT, name=name, step=step, budget_s=budget_s)
    r = subprocess.run([sys.executable, "-c", script], capture_output=True, text=True, env=env, timeout=900, cwd=ROOT)
    if r.returncode != 0:
        raise RuntimeError(r.stderr[-2000:])
    t, n = r.stdout.strip().splitlines()[-1].split()
    return float(t), int(n)


def run_reference(args, rank, world):
    if rank != 0:
        return None
    if WORKLOADS[args.workload].get("kind") == "sweep":
        # the oracle cannot assemble the sweep's larger instances within a bounded
        # sample: each instance's request is extrapolated from the sampled solve at
        # its middle frequency, once, and the sweep is their sum over the frequencies
        W = WORKLOADS[args.workload]
        cat, khat, _ = sweep_catalogue(W)
        total, spent = 0.0, 0.0
        for i, c in enumerate(cat):
            t, sample1, _, sp = oracle_step_seconds(f"{args.workload}-inst{i}", 0, quick=True)
            total += t * len(c["freqs"])
            spent += sp
        nrhs = len(khat) * sum(len(c["freqs"]) for c in cat)
        v = nrhs / total
        sample = ("per instance, the sampled oracle solve of one request at its middle frequency (" + sample1 +
                  "), times its frequencies; measured once for the run")
        return {
            "impl": "reference", "metric": METRIC, "value": v, "unit": "solves/s", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * total, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "c128", "data": "synthetic",
            "config": {"workload": args.workload, "parallelism": "host cores"}, "extrapolated": True,
            "cpu_baseline": {"value": v, "unit": "solves/s", "cores": 1, "kind": "oracle", "sample": sample,
                             "extrapolated": True, "sampled_s": spent, "cpu": cpu_model(), "nproc": os.cpu_count()},
            "e2e": {"value": v, "unit": "solves/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
        }
    if WORKLOADS[args.workload].get("kind") == "serving":
        spent, rhs, times = 0.0, 0, []
        for i in range(args.warmup + args.steps):
            t, n = oracle_serving(args.workload, i, budget_s=10.0 if i < args.warmup else 20.0)
            if i >= args.warmup:
                spent += t
                rhs += n
                times.append(t / max(n, 1))
        v = rhs / spent
        sample = ("the oracle on each timed step's requests (serving: the trace in arrival order; sweep: the "
                  "(instance, frequency) pairs of the instances up to 1,280 triangles in a seeded random order) "
                  "with dense assembly, LU, one back substitution per plane wave, no operator cache, until 20 s "
                  "were spent; single thread")
        return {
            "impl": "reference", "metric": METRIC, "value": v, "unit": "solves/s", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * spent / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "c128", "data": "synthetic",
            "config": {"workload": args.workload, "parallelism": "host cores"}, "extrapolated": False,
            "cpu_baseline": {"value": v, "unit": "solves/s", "cores": 1, "kind": "oracle", "sample": sample,
                             "sampled_s": spent, "cpu": cpu_model(), "nproc": os.cpu_count()},
            "e2e": {"value": v, "unit": "solves/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
        }
    times, spent = [], 0.0
    sample, extrap = None, False
    for i in range(args.warmup + args.steps):
        t, sample, extrap, sp = oracle_step_seconds(args.workload, i, quick=True)
        spent += sp
        if i >= args.warmup:
            times.append(t)
    total = sum(times)
    # the oracle's dense LU serves every right-hand side of a request
    v = args.steps * _nrhs(WORKLOADS[args.workload]) / total
    return {
        "impl": "reference", "metric": METRIC,
        "value": v, "unit": "solves/s", "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": 1e3 * total / args.steps, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "c128", "data": "synthetic",
        "config": {"workload": args.workload, "parallelism": "host cores"},
        "extrapolated": extrap,
        "latency_ms": {"p50": 1e3 * float(np.percentile(times, 50)), "p99": 1e3 * float(np.percentile(times, 99))},
        "cpu_baseline": {"value": v, "unit": "solves/s", "cores": 1, "kind": "oracle", "sample": sample,
                         "extrapolated": extrap, "sampled_s": spent, "cpu": cpu_model(), "nproc": os.cpu_count()},
        "e2e": {"value": v, "unit": "solves/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default=DEFAULT_WORKLOAD, choices=sorted(WORKLOADS))
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true", help="skip the host-buffer end-to-end leg (profiling runs)")
    args = ap.parse_args()
    args.warmup = max(args.warmup, 3)
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    if world > 1:
        import torch
        torch.distributed.init_process_group("nccl" if args.impl == "ours" else "gloo")
    if args.impl == "reference":
        out = run_reference(args, rank, world)
    elif WORKLOADS[args.workload].get("kind") == "serving":
        out = run_serving(args, rank, world)
    elif WORKLOADS[args.workload].get("kind") == "sweep":
        out = run_sweep(args, rank, world)
    else:
        out = run_ours(args, rank, world)
        if rank == 0 and world == 1 and not args.no_cpu_baseline:
            nr = _nrhs(WORKLOADS[args.workload])
            fi = len(_freqs(WORKLOADS[args.workload])) // 2
            try:
                t, sample, extrap, spent = oracle_step_seconds(args.workload, fi)
                out["cpu_baseline"] = {"value": nr / t, "unit": "solves/s", "cores": 1, "kind": "oracle",
                                       "sample": sample, "extrapolated": extrap, "sampled_s": spent,
                                       "cpu": cpu_model(), "nproc": os.cpu_count()}
            except Exception as e:  # the GPU line stands without it
                out["cpu_baseline"] = {"value": None, "unit": "solves/s", "cores": 1, "kind": "oracle",
                                       "error": str(e).strip().splitlines()[-1][:300]}
            try:
                ncores = os.cpu_count() or 1
                rate, wall = oracle_all_cores(args.workload, fi, ncores)
                out["cpu_baseline_all_cores"] = {
                    "value": nr * rate, "unit": "solves/s", "cores": ncores, "kind": "oracle",
                    "sample": f"{ncores} single-threaded copies of the sampled solve at once (the quick sample of "
                              "the reference arm), aggregate rate", "extrapolated": not args.workload.startswith("sphere"),
                    "sampled_s": wall}
            except Exception as e:
                out["cpu_baseline_all_cores"] = {"value": None, "error": str(e).strip().splitlines()[-1][:300]}
    if rank == 0 and out is not None:
        print(json.dumps(out))
    if world > 1:
        import torch
        torch.distributed.destroy_process_group()


if __name__ == "__main__":
    main()
