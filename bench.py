"""Throughput of the fused D3Q19 BGK stream-collide path on GB300.

One step = one fused stream-collide update of the whole lattice (one kernel
launch). The workload is the walled channel: 256 x 128 x 128 cells, periodic
in x, solid walls at y in {0, 127} and z in {0, 127}, seeded spherical
obstacles (radius 3-6) filling 10% of the interior, halfway bounce-back,
uniform body force g_x = 1e-6, tau = 0.55, populations stored in FP32.
Synthetic inputs (lbm_inputs); the lattices (2 x 319 MB) exceed L2, so no
flush is needed between steps.

Prints one JSON line: value = million fluid-cell updates per second (MFLUPS,
the paper's metric), the roofline of the step kernel against measured HBM
bandwidth, the FP64 oracle timed on the host cores beside the host copy
bandwidth, an end-to-end figure through host buffers, the other storage
formats and the adjoint/forward step-time ratio on the same workload, the
512^3 Taylor-Green box in every format and pattern, and the cost of a z-slab
halo exchange on that box. The K timed steps run as 5 back-to-back
sub-regions (median and spread of the step time beside the whole-region
value); every other leg is timed as 5 repetitions of at least 10 ms each.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]

With N > 1 (torchrun), every rank runs an independent replica on its own GPU
(weak scaling; the method needs no exchange between replicas); rank 0 prints
the aggregate over the max-over-ranks time. With --decompose z the ranks
instead share one lattice as z-slabs, exchanging halos every step over the
process group (strong scaling).
"""
import argparse
import hashlib
import glob
import json
import os
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import lbm_inputs  # noqa: E402

METRIC = "D3Q19 MLUPS & % of HBM roofline per precision; adjoint/forward step-time ratio"
NX, NY, NZ, TAU, GX, SOLID = 256, 128, 128, 0.55, 1e-6, 0.10
WORKLOAD = ("D3Q19 BGK channel 256x128x128 (x periodic), walls y=0/127 z=0/127 + seeded spheres r 3-6 "
            "(10% solid), halfway bounce-back, g_x=1e-6, tau=0.55")
# algorithmic bytes per fluid-cell update: 19 loads + 19 stores of the stored
# value; the moment-split formats also read and write one 8-byte momentum word
PDF_BYTES = {"f64": 304, "f32": 152, "f16s": 76, "bf16s": 76, "f16m": 92, "bf16m": 92}
FLAG_BYTES = 1
STEP_KERNEL = "k_step"


def measured_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            p = json.load(f)
        return float(p["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


def kernel_source_hash():
    """Hash of the sources the two-grid step kernels and their launch
    configuration are built from: the device, launch and kernel headers, the
    per-format kernel units, the context setup (launch shape, masks, links)
    and the C header. The AA, reverse-step, halo and allocation-free units do
    not enter the step kernels and are left out."""
    csrc = os.path.join(ROOT, "paper_1112_0850_gb300", "csrc")
    files = [os.path.join(csrc, n) for n in ("lbm_device.cuh", "lbm_launch.h", "lbm_kernels.cuh", "lbm_capi.cu",
                                              "lbm_setup.cu")]
    files += sorted(glob.glob(os.path.join(csrc, "lbm_ops_*.cu")))
    files.append(os.path.join(ROOT, "include", "lbm_capi.h"))
    h = hashlib.sha256()
    for p in files:
        with open(p, "rb") as f:
            h.update(os.path.basename(p).encode())
            h.update(f.read())
    return h.hexdigest()[:16]


def ncu_traffic(case, storage):
    """DRAM bytes (read + write) of one step launch from the committed ncu
    summary, if it was taken on the current kernel sources; else None."""
    path = os.path.join(ROOT, "profiles", "step_kernel_traffic.json")
    try:
        with open(path) as f:
            d = json.load(f)
    except Exception:
        return None
    if d.get("src_hash") != kernel_source_hash():
        return None
    ent = d.get("kernels", {}).get("%s/%s" % (case, storage))
    return None if ent is None else float(ent["dram_bytes_per_launch"])


def record_traffic(pairs):
    """Write profiles/step_kernel_traffic.json from ncu reports: for each
    KEY=REPORT (KEY as in ncu_traffic, e.g. channel/f32), the DRAM bytes read
    and written by the one captured launch in REPORT, stamped with the hash of
    the kernel sources they were taken on. Reads the reports with `ncu -i`;
    needs no GPU."""
    import csv
    import io
    import subprocess
    entries = {}
    for arg in pairs:
        key, rep = arg.split("=", 1)
        out = subprocess.run(["ncu", "-i", rep, "--page", "raw", "--csv"], capture_output=True, text=True,
                             check=True).stdout
        rows = list(csv.reader(io.StringIO(out)))
        hdr, units, vals = rows[0], rows[1], rows[2]

        def get(name):
            i = hdr.index(name)
            scale = {"byte": 1, "Kbyte": 1e3, "Mbyte": 1e6, "Gbyte": 1e9}.get(units[i], 1)
            return float(vals[i].replace(",", "")) * scale

        r, w = get("dram__bytes_read.sum"), get("dram__bytes_write.sum")
        entries[key] = {"dram_bytes_per_launch": r + w, "dram_read": r, "dram_write": w,
                        "kernel": vals[hdr.index("Kernel Name")], "report": os.path.basename(rep)}
    out = {"src_hash": kernel_source_hash(), "kernels": entries,
           "note": "one cold-cache ncu launch of each kernel; writes still dirty in L2 at kernel end are not counted"}
    with open(os.path.join(ROOT, "profiles", "step_kernel_traffic.json"), "w") as f:
        json.dump(out, f, indent=1)
    print(json.dumps(out, indent=1))


def workload_flags():
    return lbm_inputs.channel_flags(NX, NY, NZ, SOLID, lbm_inputs.seed_for(1))


class ClockSampler:
    """nvidia-smi SM clock and throttle reasons sampled every 100 ms."""
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.path = None

    def __enter__(self):
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), "--query-gpu=" + self.FIELDS,
                                          "--format=csv,noheader,nounits", "-lms", "100"],
                                         stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None
        time.sleep(0.3)
        return self

    def __exit__(self, *a):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()

    def summary(self):
        rows = []
        try:
            for line in open(self.path):
                parts = [p.strip() for p in line.split(",")]
                if len(parts) >= 9:
                    rows.append(parts)
        except Exception:
            pass
        if self.path and os.path.exists(self.path):
            os.unlink(self.path)
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no nvidia-smi samples"], "samples": 0}

        def num(v):
            try:
                return float(v)
            except ValueError:
                return float("nan")

        sm = np.array([num(r[1]) for r in rows])
        mx = np.array([num(r[2]) for r in rows])
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[k] for r in rows for k in range(4) if r[5 + k].lower() == "active"})
        return {"sm_mhz": float(np.nanmedian(sm)), "sm_max_mhz": float(np.nanmax(mx)), "reasons": reasons,
                "samples": len(rows), "power_w_max": float(np.nanmax([num(r[3]) for r in rows]))}


# ----------------------------------------------------------------------------------------------
def oracle_baseline(flags, budget_s, threads=None):
    """Time the FP64 oracle on a z-slab sample of the workload: returns
    (MFLUPS, cores, sample description, fluid cells, steps)."""
    import oracle
    cores = threads or oracle.max_threads()

    def slab(nzs):
        z0 = (NZ - nzs) // 2
        fl = np.ascontiguousarray(flags[z0:z0 + nzs])
        f = oracle.init_equilibrium(np.zeros((3, nzs, NY, NX)), flags=fl)
        return fl, f

    # calibrate with one step of the whole channel (OpenMP over z needs the
    # layers to use every core), then take as many steps as fill the budget,
    # or a thinner slab if one step already exceeds it
    fl, f = slab(NZ)
    Fg = np.array([GX, 0.0, 0.0])
    f = oracle.run(f, TAU, 1, flags=fl, F=Fg, threads=cores)  # first touch, thread start-up
    t0 = time.perf_counter()
    oracle.run(f, TAU, 4, flags=fl, F=Fg, threads=cores)  # (each call allocates its scratch lattice)
    t_step = (time.perf_counter() - t0) / 4
    if 2 * t_step <= budget_s:
        nzs, steps = NZ, int(budget_s / t_step)
    else:
        nzs, steps = int(max(1, NZ * budget_s / (2 * t_step))), 2
    fl, f = slab(nzs)
    nfl = int((fl == 0).sum())
    t0 = time.perf_counter()
    oracle.run(f, TAU, steps, flags=fl, F=np.array([GX, 0.0, 0.0]), threads=cores)
    dt = time.perf_counter() - t0
    desc = ("oracle (plain C, FP64, OpenMP over z) on the middle %d of 128 z-layers of the channel "
            "(%dx%dx%d, %d fluid cells), %d steps, %.1f s" % (nzs, NX, NY, nzs, nfl, steps, dt))
    return nfl * steps / dt / 1e6, cores, desc, nfl, steps


def reference_arm(args):
    """The oracle as the reference implementation: each step one oracle update
    of a z-slab sample of the workload, sized so the whole run stays short."""
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    import oracle
    flags = workload_flags()
    cores = oracle.max_threads()
    nsteps = args.steps + args.warmup
    fl4 = np.ascontiguousarray(flags[62:66])
    f = oracle.init_equilibrium(np.zeros((3, 4, NY, NX)), flags=fl4)
    t0 = time.perf_counter()
    oracle.run(f, TAU, 1, flags=fl4, F=np.array([GX, 0.0, 0.0]), threads=cores)
    t_cell = (time.perf_counter() - t0) / (4 * NY * NX)
    budget = 120.0
    nzs = int(max(2, min(NZ, budget / max(t_cell, 1e-12) / (NY * NX) / max(nsteps, 1))))
    z0 = (NZ - nzs) // 2
    fl = np.ascontiguousarray(flags[z0:z0 + nzs])
    nfl = int((fl == 0).sum())
    f = oracle.init_equilibrium(np.zeros((3, nzs, NY, NX)), flags=fl)
    F = np.array([GX, 0.0, 0.0])
    f = oracle.run(f, TAU, args.warmup, flags=fl, F=F, threads=cores)
    t0 = time.perf_counter()
    oracle.run(f, TAU, args.steps, flags=fl, F=F, threads=cores)
    dt = time.perf_counter() - t0
    value = nfl * args.steps / dt / 1e6
    sample = ("each step: one oracle update (plain C, FP64, OpenMP over z) of the middle %d of 128 z-layers "
              "of the channel (%dx%dx%d, %d fluid cells)" % (nzs, NX, NY, nzs, nfl))
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": "MFLUPS", "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": dt / max(args.steps, 1) * 1e3,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": {"workload": WORKLOAD, "storage": "f64 (oracle)",
                                            "parallelism": "host cores"},
            "cpu_baseline": {"value": value, "unit": "MFLUPS", "cores": cores, "kind": "oracle", "sample": sample},
            "e2e": {"value": value, "unit": "MFLUPS", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


# ----------------------------------------------------------------------------------------------
def max_over_ranks(v, world, device):
    """Largest value of v over all ranks (the slowest replica's time)."""
    if world == 1:
        return v
    import torch
    import torch.distributed as dist
    t = torch.tensor([float(v)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return t.item()


def aggregate_mflups(units_per_rank, world, seconds):
    """Whole-job throughput: every rank processed units_per_rank in at most `seconds`."""
    return world * units_per_rank / seconds / 1e6


def time_steps(torch, lat, steps, warmup):
    """Warm up, then time `steps` single-step launches with CUDA events on the lattice's stream."""
    lat.step(warmup)
    st = lat.stream
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    e0.record(st)
    lat.step(steps)
    e1.record(st)
    torch.cuda.synchronize()
    return e0.elapsed_time(e1) / 1e3


REPS = 5          # repetitions of every timed region (median and spread reported)
MIN_REP_S = 0.01  # device time of one repetition of a leg, at least (so >= 50 ms a leg)


def time_reps(torch, stream, run, reps=REPS):
    """Enqueue run() `reps` times back to back on `stream`, with a CUDA event
    between repetitions; return the device seconds of each repetition."""
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(reps + 1)]
    torch.cuda.synchronize()
    ev[0].record(stream)
    for k in range(reps):
        run()
        ev[k + 1].record(stream)
    torch.cuda.synchronize()
    return [ev[k].elapsed_time(ev[k + 1]) / 1e3 for k in range(reps)]


def spread(per_step):
    """Median, min, max and relative spread of per-step times (seconds)."""
    v = sorted(per_step)
    med = v[len(v) // 2]
    return {"median_ms": med * 1e3, "min_ms": v[0] * 1e3, "max_ms": v[-1] * 1e3,
            "spread": (v[-1] - v[0]) / med, "reps": len(v)}


def leg(torch, lat, warmup=3):
    """Time a lattice's steps: REPS repetitions of k steps each, k chosen so a
    repetition takes at least MIN_REP_S of device time (one untimed repetition
    first, which also captures the step graph where k >= 32). Returns
    (median seconds per step, spread record)."""
    lat.step(warmup)
    t1 = time_steps(torch, lat, 2, 0) / 2
    k = max(2, int(np.ceil(MIN_REP_S / max(t1, 1e-9))))
    lat.step(k)
    ts = time_reps(torch, lat.stream, lambda: lat.step(k))
    rec = spread([t / k for t in ts])
    rec["steps_per_rep"] = k
    return rec["median_ms"] / 1e3, rec


def host_copy_gbs(cores, nbytes=1 << 30, reps=5):
    """Host copy bandwidth (STREAM copy: bytes read + bytes written per second)
    with torch's multithreaded CPU copy over `cores` threads, best of reps."""
    import torch
    torch.set_num_threads(cores)
    a = torch.ones(nbytes // 8, dtype=torch.float64)
    b = torch.empty_like(a)
    b.copy_(a)
    best = float("inf")
    for _ in range(reps):
        t0 = time.perf_counter()
        b.copy_(a)
        best = min(best, time.perf_counter() - t0)
    return 2 * nbytes / best / 1e9


def sweep():
    """Throughput against domain size (periodic n^3 boxes, the paper's domain
    sweeps, Sec. 7) and the effect of padding rows to 128 bytes (Sec. 6): MLUPS
    and fraction of the measured copy bandwidth per case."""
    import torch
    from paper_1112_0850_gb300 import build
    from paper_1112_0850_gb300.lattice import Lattice
    build.build()
    peak, _ = measured_peaks()

    def run(n, storage, row_align=0):
        lat = Lattice(n, n, n, 0.6, storage=storage, row_align=row_align)
        rng = np.random.default_rng(1)
        u = torch.tensor(0.01 * rng.standard_normal((3, n, n, n)), dtype=lat.real).cuda()
        lat.init_equilibrium(u)
        t, rec = leg(torch, lat, 5)
        pitch = lat.info.pitch
        lat.close()
        gbs = n ** 3 * PDF_BYTES[storage] / t / 1e9
        return {"n": n, "storage": storage, "pitch": pitch, "mlups": n ** 3 / t / 1e6, "gbs": gbs,
                "frac": gbs / peak, "timing": rec}

    sizes = [16, 24, 32, 48, 64, 96, 128, 160, 200, 256, 320, 384, 448, 512]
    with ClockSampler(torch.cuda.current_device()) as clk:
        res = [run(n, s) for s in ("f32", "f16s", "bf16m") for n in sizes]
        pad = [run(n, s, ra) for s in ("f32", "f16s") for n in (200, 250) for ra in (0, 128)]
    out = {"sweep": res, "padding": pad, "clocks": clk.summary(),
           "note": "periodic boxes, random velocities (0.01), tau 0.6; small boxes fit in the 129 MB L2, so "
                   "their fraction of HBM copy bandwidth can exceed 1; padding: row_align 128 = the paper's "
                   "128-byte rows, 0 = rows padded only to a pair of cells (the default)"}
    print(json.dumps(out), flush=True)


def decomposed(args, torch, dist, world, rank):
    """One lattice split over the ranks as z-slabs (slabs.RankSlab): every step
    exchanges the five crossing populations of each face with the neighbouring
    ranks (point-to-point; NCCL between GPUs, a local copy on one rank), then
    steps the slab. value = the whole lattice's fluid-cell updates per second
    (strong scaling: the lattice is fixed, each rank holds 1/N of it)."""
    from paper_1112_0850_gb300.slabs import RankSlab
    if world == 1:  # a one-rank process group for RankSlab (its exchange is then a local copy)
        import socket
        sck = socket.socket()
        sck.bind(("127.0.0.1", 0))
        port = sck.getsockname()[1]
        sck.close()
        dist.init_process_group("gloo", init_method="tcp://127.0.0.1:%d" % port, rank=0, world_size=1)
    storage = args.storage
    if args.case == "channel":
        flags = workload_flags()
        sl = RankSlab(NX, NY, NZ, TAU, flags=flags, force=(GX, 0.0, 0.0), storage=storage)
        sl.init_equilibrium(torch.zeros((3, NZ, NY, NX), dtype=sl.lat.real))
        n_units = int((flags == 0).sum())
        workload = WORKLOAD
    else:
        n = args.n
        sl = RankSlab(n, n, n, 0.52, storage=storage)
        rho_tg, u_tg = lbm_inputs.taylor_green(n, 0.02, dtype=np.float32)
        real = torch.float64 if storage == "f64" else torch.float32
        sl.init_equilibrium(torch.from_numpy(u_tg).to(real), torch.from_numpy(rho_tg).to(real))
        del rho_tg, u_tg
        n_units = n ** 3
        workload = "D3Q19 BGK Taylor-Green vortex, periodic %d^3, U0=0.02, tau=0.52" % n
    sl.step(args.warmup)
    torch.cuda.synchronize()
    dist.barrier()
    with ClockSampler(torch.cuda.current_device()) as clk:
        ts = time_reps(torch, sl.stream, lambda: sl.step(max(1, args.steps // REPS)))
    dist.barrier()
    steps = REPS * max(1, args.steps // REPS)
    dt = max_over_ranks(sum(ts), world, "cuda")
    tot = sl.totals()
    status = sl.lat.status_word()
    slab_planes = sl.z1 - sl.z0
    sl.close()
    if rank == 0:
        line = {"metric": METRIC, "value": n_units * steps / dt / 1e6, "unit": "MFLUPS" if args.case == "channel"
                else "MLUPS", "n_gpus": world, "steps": steps, "warmup": args.warmup,
                "ms_per_step": dt / steps * 1e3, "higher_is_better": True, "scaling": "strong", "vs_baseline": None,
                "dtype": "f64" if storage == "f64" else "f32", "data": "synthetic",
                "config": {"workload": workload, "storage": storage, "decomposition": "z-slabs, one per rank",
                           "planes_per_rank": slab_planes,
                           "parallelism": "z-slabs over %d ranks, point-to-point halo exchange per step" % world},
                "timing": spread([t / max(1, args.steps // REPS) for t in ts]), "clocks": clk.summary(),
                "mass": float(tot[0]), "status_word": status, "gpu_launches": None}
        print(json.dumps(line), flush=True)
    dist.destroy_process_group()


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5000)
    ap.add_argument("--warmup", type=int, default=20)
    ap.add_argument("--impl", default="gb300", choices=["gb300", "reference"])
    ap.add_argument("--no-extras", action="store_true", help="skip other precisions, adjoint ratio, CPU baseline")
    ap.add_argument("--case", default="channel", choices=["channel", "taylor-green"],
                    help="headline workload: the walled channel (default) or a periodic Taylor-Green box")
    ap.add_argument("--storage", default="f32", choices=["f64", "f32", "f16s", "bf16s", "f16m", "bf16m"])
    ap.add_argument("--n", type=int, default=512, help="Taylor-Green box edge")
    ap.add_argument("--pattern", default="pull", choices=["pull", "aa"],
                    help="two lattices (pull) or one lattice updated in place (AA pattern)")
    ap.add_argument("--sweep", action="store_true",
                    help="domain-size sweep of periodic boxes and the row-padding ablation (one JSON line)")
    ap.add_argument("--adjoint-only", type=int, default=0, metavar="K",
                    help="run K recorded steps, the seed and K reverse steps on the channel (for profilers) and exit")
    ap.add_argument("--record-traffic", nargs="+", metavar="KEY=REPORT",
                    help="write profiles/step_kernel_traffic.json from ncu reports and exit")
    ap.add_argument("--decompose", choices=["z"], default=None,
                    help="split one lattice over the ranks as z-slabs with a halo exchange per step "
                         "(strong scaling), instead of independent replicas")
    args = ap.parse_args()
    if args.record_traffic:
        return record_traffic(args.record_traffic)
    args.warmup = max(3, args.warmup)
    if args.impl == "reference":
        return reference_arm(args)
    if args.sweep:
        return sweep()

    import torch
    import torch.distributed as dist
    from paper_1112_0850_gb300 import build
    from paper_1112_0850_gb300.lattice import Lattice

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    torch.cuda.set_device(local)
    if world > 1 and rank != 0:
        dist.barrier()  # rank 0 builds (if anything is out of date), the others then load
    build.build()
    if world > 1 and rank == 0:
        dist.barrier()

    def barrier():
        if world > 1:
            dist.barrier()

    if args.decompose:
        return decomposed(args, torch, dist, world, rank)

    flags = workload_flags()
    F = (GX, 0.0, 0.0)
    storage = args.storage
    if args.adjoint_only:
        # the reverse step alone, for profilers: K recorded steps, seed, K reverse steps
        K = args.adjoint_only
        lat = Lattice(NX, NY, NZ, TAU, flags=flags, force=F, storage=storage)
        lat.init_equilibrium(lat.zeros(3))
        tape = lat.new_tape(K)
        gF = lat.zeros(3)
        lat.step(args.warmup)
        lat.step_record(K, tape)
        lat.adjoint_seed(lat.zeros(3).add_(1e-3), None, gF)
        lat.adjoint_step(K, tape, gF)
        torch.cuda.synchronize()
        status = lat.status_word()
        lat.close()
        print(json.dumps({"adjoint_only": K, "storage": storage, "status_word": status}), flush=True)
        return 0 if status == 0 else 1
    if args.case == "channel":
        lat = Lattice(NX, NY, NZ, TAU, flags=flags, force=F, storage=storage, pattern=args.pattern)
        lat.init_equilibrium(lat.zeros(3))
        n_cells = NX * NY * NZ
        workload = WORKLOAD
        flag_bytes = FLAG_BYTES
    else:
        n = args.n
        lat = Lattice(n, n, n, 0.52, storage=storage, pattern=args.pattern)
        rho_tg, u_tg = lbm_inputs.taylor_green(n, 0.02, dtype=np.float32)
        real = torch.float64 if storage == "f64" else torch.float32
        lat.init_equilibrium(torch.from_numpy(u_tg).to("cuda", real), torch.from_numpy(rho_tg).to("cuda", real))
        del rho_tg, u_tg
        n_cells = n ** 3
        workload = "D3Q19 BGK Taylor-Green vortex, periodic %d^3, U0=0.02, tau=0.52" % n
        flag_bytes = 0
    n_fluid = lat.n_fluid

    # ---- headline: K steps, device-resident ------------------------------------------
    # The K timed steps run as REPS back-to-back sub-regions with a CUDA event
    # between them: `value` is K steps over the whole region, and the
    # sub-regions give the median and spread of the step time.
    # The clock sampler starts first: its start leaves the GPU idle for 0.3 s,
    # which the warm-up then follows straight before the timed region.
    chunks = [args.steps // REPS + (1 if k < args.steps % REPS else 0) for k in range(REPS)]
    chunks = [c for c in chunks if c > 0]
    for c in set(chunks):  # capture the sub-regions' step graphs (host work; no step runs)
        lat.prepare_steps(c)
    with ClockSampler(torch.cuda.current_device()) as clk:
        lat.step(args.warmup)
        torch.cuda.synchronize()
        barrier()
        it = iter(chunks)
        ts = time_reps(torch, lat.stream, lambda: lat.step(next(it)), reps=len(chunks))
    barrier()
    dt_local = sum(ts)
    dt = max_over_ranks(dt_local, world, "cuda")
    clocks = clk.summary()
    status = lat.status_word()
    value = aggregate_mflups(n_fluid * args.steps, world, dt)
    per_launch = dt_local / args.steps
    head_spread = spread([t / c for t, c in zip(ts, chunks)])
    peak, peak_kind = measured_peaks()
    alg_bytes = n_fluid * PDF_BYTES[storage] + n_cells * flag_bytes
    achieved = alg_bytes / per_launch / 1e9
    traffic = ncu_traffic(args.case if args.case == "channel" else "taylor-green-%d" % args.n, storage)

    extras = {}
    cpu = None
    e2e = None
    if not args.no_extras and args.case == "channel" and storage == "f32":
        # ---- other storage formats on the same workload -------------------------------------
        per_prec = {"f32": {"mflups": n_fluid / per_launch / 1e6, "gbs": achieved, "frac": achieved / peak,
                            "bytes_per_lup": PDF_BYTES["f32"], "timing": head_spread}}
        for s in ("f64", "f16s", "bf16s", "f16m", "bf16m"):
            l2 = Lattice(NX, NY, NZ, TAU, flags=flags, force=F, storage=s)
            l2.init_equilibrium(l2.zeros(3))
            t, rec = leg(torch, l2, args.warmup)
            gbs = (n_fluid * PDF_BYTES[s] + n_cells * FLAG_BYTES) / t / 1e9
            per_prec[s] = {"mflups": n_fluid / t / 1e6, "gbs": gbs, "frac": gbs / peak, "bytes_per_lup": PDF_BYTES[s],
                           "timing": rec}
            l2.close()
        extras["per_precision"] = per_prec
        # ---- the 512^3 periodic Taylor-Green box, every storage format -----------------
        tg = {}
        n = 512
        rho_tg, u_tg = lbm_inputs.taylor_green(n, 0.02, dtype=np.float32)
        rho_tg, u_tg = torch.from_numpy(rho_tg).cuda(), torch.from_numpy(u_tg).cuda()
        for s in ("f32", "f16s", "bf16s", "f16m", "bf16m", "f64"):
            l2 = Lattice(n, n, n, 0.52, storage=s)
            if s == "f64":
                l2.init_equilibrium(u_tg.double(), rho_tg.double())
            else:
                l2.init_equilibrium(u_tg, rho_tg)
            t, rec = leg(torch, l2)
            gbs = n ** 3 * PDF_BYTES[s] / t / 1e9
            tg[s] = {"mlups": n ** 3 / t / 1e6, "gbs": gbs, "frac": gbs / peak, "ms_per_step": t * 1e3,
                     "bytes_per_lup": PDF_BYTES[s], "timing": rec}
            l2.close()
        extras["taylor_green_512"] = tg
        # ---- the AA pattern (one lattice, in place) on both workloads ------------------
        aa = {}
        for s in ("f32", "f16s", "bf16s"):
            l2 = Lattice(n, n, n, 0.52, storage=s, pattern="aa")
            l2.init_equilibrium(u_tg, rho_tg)
            t, rec = leg(torch, l2, 4)
            gbs = n ** 3 * PDF_BYTES[s] / t / 1e9
            aa["taylor_green_512_" + s] = {"mlups": n ** 3 / t / 1e6, "gbs": gbs, "frac": gbs / peak, "timing": rec}
            l2.close()
        for s in ("f32", "f16s"):
            l2 = Lattice(NX, NY, NZ, TAU, flags=flags, force=F, storage=s, pattern="aa")
            l2.init_equilibrium(l2.zeros(3))
            t, rec = leg(torch, l2, args.warmup)
            gbs = (n_fluid * PDF_BYTES[s] + n_cells * FLAG_BYTES) / t / 1e9
            aa["channel_" + s] = {"mflups": n_fluid / t / 1e6, "gbs": gbs, "frac": gbs / peak, "timing": rec}
            l2.close()
        extras["aa_pattern"] = aa
        # ---- the 512^3 box as two z-slabs on this GPU: what the halo exchange costs ---------
        from paper_1112_0850_gb300.slabs import SlabSet
        sl = SlabSet(n, n, n, 0.52, 2, storage="f32")
        sl.init_equilibrium(u_tg, rho_tg)
        t_sl, rec_sl = leg(torch, sl)  # an exchange, then a step of each slab
        for _ in range(3):
            sl.exchange()
        ts_ex = time_reps(torch, sl.stream, lambda: [sl.exchange() for _ in range(20)])
        t_ex = spread([t / 20 for t in ts_ex])["median_ms"] / 1e3
        face = 5 * n * n * 4  # five FP32 populations of one 512^2 plane
        sl.overlap = True  # the exchange on a second stream while the interior planes update
        t_ov, rec_ov = leg(torch, sl)
        extras["z_slabs"] = {
            "workload": "Taylor-Green 512^3 FP32 as 2 z-slabs of 256 planes plus 2 ghost planes each",
            "mlups": n ** 3 / t_sl / 1e6, "exchange_us": t_ex * 1e6, "face_bytes": face,
            "exchange_gbs": 16 * face / t_ex / 1e9, "exchange_share_of_step": t_ex / t_sl,
            "mlups_overlapped": n ** 3 / t_ov / 1e6, "timing": rec_sl, "timing_overlapped": rec_ov}
        sl.close()
        del rho_tg, u_tg
        # ---- adjoint / forward step-time ratio (FP32, per-cell force gradient) -------------
        K = 100
        tape = lat.new_tape(K)
        gF = lat.zeros(3)
        lat.adjoint_seed(lat.zeros(3).add_(1e-3), None, gF)
        st = lat.stream
        lat.step_record(K, tape)
        lat.adjoint_step(K, tape, gF)
        ratios, ratios_nr, t_adjs = [], [], []
        for _ in range(REPS):
            ev = [torch.cuda.Event(enable_timing=True) for _ in range(3)]
            torch.cuda.synchronize()
            ev[0].record(st)
            lat.step_record(K, tape)
            ev[1].record(st)
            lat.adjoint_step(K, tape, gF)
            ev[2].record(st)
            torch.cuda.synchronize()
            t_rec = ev[0].elapsed_time(ev[1]) / 1e3 / K
            t_adj = ev[1].elapsed_time(ev[2]) / 1e3 / K
            ratios.append((t_rec + t_adj) / head_spread["median_ms"] * 1e3)
            ratios_nr.append(t_adj / head_spread["median_ms"] * 1e3)
            t_adjs.append(t_adj)
        ratios.sort()
        ratios_nr.sort()
        t_adj = sorted(t_adjs)[REPS // 2]
        extras["adjoint_forward_ratio"] = ratios[REPS // 2]
        extras["adjoint_forward_ratio_no_recompute"] = ratios_nr[REPS // 2]
        extras["adjoint_forward_ratio_range"] = [ratios[0], ratios[-1]]
        extras["adjoint_step_gbs"] = (n_fluid * (76 + 76 + 16 + 24) + n_cells) / t_adj / 1e9
        extras["adjoint_timing"] = dict(spread(t_adjs), steps_per_rep=K)
        del tape, gF
        # ---- end to end through the C-ABI with host buffers --------------------------------
        u0_host = torch.zeros((3, NZ, NY, NX), dtype=torch.float32).pin_memory()
        u_host = torch.empty((3, NZ, NY, NX), dtype=torch.float32).pin_memory()
        rho_host = torch.empty((NZ, NY, NX), dtype=torch.float32).pin_memory()
        torch.cuda.synchronize()
        barrier()
        t0 = time.perf_counter()
        l3 = Lattice(NX, NY, NZ, TAU, flags=flags, force=F, storage="f32")
        l3.init_equilibrium(u0_host)
        l3.step(args.steps)
        l3.macros(rho_host, u_host)
        sums = l3.reduce()
        l3.close()
        t_e2e = max_over_ranks(time.perf_counter() - t0, world, "cuda")
        h2d = flags.nbytes + u0_host.numel() * 4
        d2h = u_host.numel() * 4 + rho_host.numel() * 4 + 32
        e2e = {"value": aggregate_mflups(n_fluid * args.steps, world, t_e2e), "unit": "MFLUPS",
               "h2d_bytes_per_step": h2d / args.steps, "d2h_bytes_per_step": d2h / args.steps,
               "what": "whole job per replica: lbm_create from host flags, init from pinned host u0, "
                       "%d steps, macros and FP64 totals back to host, destroy" % args.steps,
               "mass": float(sums[0])}
        # ---- CPU baseline: the oracle on a bounded sample -----------------------------------
        if rank == 0 and world == 1:
            v, cores, desc, _, _ = oracle_baseline(flags, 10.0)
            copy = host_copy_gbs(cores)
            cpu = {"value": v, "unit": "MFLUPS", "cores": cores, "kind": "oracle", "sample": desc,
                   "host_copy_gbs": copy,
                   "host_copy_how": "torch CPU copy of 1 GiB FP64 over %d threads, read + write bytes, best of 5" % cores,
                   "host_model_mflups_fp64": copy * 1e3 / 456.0,
                   "host_model_note": "the paper's CPU model (Sec. 4): 456 B per FP64 update with write-allocate"}

    lat_bytes = lat.info.lattice_bytes
    # kernels per step in the timed region: the step kernel, plus the link
    # kernel of 16-bit shifted storage on a lattice with solid cells
    kernels_per_step = 2 if (args.pattern == "pull" and storage in ("f16s", "bf16s") and n_fluid < n_cells) else 1
    lat.close()
    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": "MFLUPS", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": dt / args.steps * 1e3, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64" if storage == "f64" else "f32",
            "data": "synthetic",
            "config": {"workload": workload, "n_cells": n_cells, "n_fluid": n_fluid,
                       "storage": storage + (" (moment split: 16-bit momentum + remainders)" if storage.endswith("m")
                                             else " (shifted f - w)"),
                       "pattern": args.pattern,
                       "l2": "no flush: the %s (%.0f MB each) exceed%s the 129 MB L2" % (
                           "lattice" if args.pattern == "aa" else "two lattices", lat_bytes / 1e6,
                           "s" if args.pattern == "aa" else ""),
                       "parallelism": "replicas" if world > 1 else "single GPU"},
            "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                         "frac": achieved / peak, "traffic": traffic,
                         "kernel": "%s<%s%s>" % (STEP_KERNEL if args.pattern == "pull" else "k_aa_even+k_aa_odd",
                                                 storage,
                                                 ",flags,uniform force" if args.case == "channel" else ""),
                         "peak_source": peak_kind + " hbm_gbs (MEASURED_PEAKS.json)",
                         "alg_bytes_per_launch": alg_bytes},
            "cpu_baseline": cpu, "e2e": e2e, "gpu_launches": args.steps * kernels_per_step, "clocks": clocks,
            "status_word": status, "timing": dict(head_spread, sub_regions=len(chunks)),
        }
        line.update(extras)
        print(json.dumps(line), flush=True)
    if world > 1:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
