"""Benchmark: two-phase lattice Boltzmann step with curved walls on the 4096^2 droplet-on-cylinder
lattice, in million fluid-node updates per second (MLUPS) and as a fraction of the measured HBM
roofline.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]

One "step" is one time step of the whole hot path: the fused step kernel over every node plus the
curved-wall pass over the boundary links.  The headline line times modified scheme B with FP32
deviation storage; "variants" times the five boundary variants (MLS, L-Bouzidi, Zhao-Yong, A, B)
in FP64 and FP32 deviation storage.  Under torchrun each rank advances its own replica of the
lattice (weak scaling, no data-path collective); rank 0 prints one JSON line.
--impl reference times the FP64 CPU oracle on the host cores instead.
"""
import argparse
import json
import os
import statistics
import subprocess
import sys
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "MLUPS and % HBM roofline per GB300; served p50/p99 latency vs plain FP64"
UNIT = "MLUPS"
SCHEME_NAMES = ("mls", "bouzidi_l", "zhao_yong", "mod_a", "mod_b")


# FP64 pipe operations (DFMA + DADD + DMUL thread instructions) per fluid-node update of the FP64
# step kernel, counted by ncu on the 2048^2 case (profiles/step_kernel_fp64_4096.md): with the
# measured FMA rate of the pipe it gives the FP64 step's ALU roofline
FP64_PIPE_OPS_PER_NODE = 128


def bytes_per_update(precision):
    # algorithmic traffic of one fluid-node update: 9 populations read + 9 written
    # (fp16_dev: the rest population in FP32, the eight moving ones in FP16)
    return {"fp64": 144, "fp32_dev": 72, "fp16_dev": 40}[precision]


# sources of the headline step kernel (step_vec_kernel, FP32 deviations); a profile summary
# records their combined sha256 prefix, so its counters are only used for the code they measured
KERNEL_SOURCES = ("step_vec.cu", "step_core.cuh", "d2q9.cuh")
PROFILE_SUMMARY = "step_vec_kernel_fp32_dev_4096.md"


def kernel_sources_sha():
    import hashlib
    h = hashlib.sha256()
    for name in KERNEL_SOURCES:
        with open(os.path.join(ROOT, "paper_1908_09235_gb300", "csrc", name), "rb") as f:
            h.update(f.read())
    return h.hexdigest()[:16]


def captured_traffic():
    """DRAM bytes per launch of the headline step kernel from the committed ncu summary, or None
    when the kernel's sources have changed since that capture."""
    import re
    summary = os.path.join(ROOT, "profiles", PROFILE_SUMMARY)
    if not os.path.exists(summary):
        return None
    text = open(summary).read()
    m_sha = re.search(r"kernel sources sha256 prefix: ([0-9a-f]+)", text)
    m_tr = re.search(r"traffic_bytes_per_launch: (\d+)", text)
    if not (m_sha and m_tr) or m_sha.group(1) != kernel_sources_sha():
        return None
    return int(m_tr.group(1))


def measured_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    return 6800.0, "fallback"


class Clocks:
    """Samples SM clocks and throttle reasons with nvidia-smi while the timed region runs."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), "--query-gpu=" + self.FIELDS,
                 "--format=csv,noheader,nounits", "-lms", "100"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except Exception:
            self.proc = None
        time.sleep(0.3)
        return self

    def __exit__(self, *a):
        self.out = ""
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.out, _ = self.proc.communicate(timeout=5)
            except Exception:
                self.proc.kill()

    def summary(self):
        rows = []
        for line in (self.out or "").splitlines():
            parts = [x.strip() for x in line.split(",")]
            if len(parts) >= 9:
                rows.append(parts)
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unavailable"]}
        sm = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        smax = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        load = [s for s in sm if s > 0.5 * max(sm)] if sm else []
        reasons = set()
        names = ("hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap")
        for r in rows:
            for name, v in zip(names, r[5:9]):
                if v.lower() == "active":
                    reasons.add(name)
        return {"sm_mhz": statistics.median(load) if load else None,
                "sm_max_mhz": max(smax) if smax else None,
                "samples": len(rows), "reasons": sorted(reasons)}


def dist_setup():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        import torch.distributed as dist
        backend = os.environ.get("LBM_BENCH_BACKEND", "nccl")
        if backend == "nccl":  # one GPU per rank, chosen before the communicator exists
            import torch
            torch.cuda.set_device(local)
        dist.init_process_group(backend)
    return world, rank, local


def max_over_ranks(x, world):
    """Maximum of a float over ranks (identity for one process)."""
    if world <= 1:
        return x
    import torch
    import torch.distributed as dist
    dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([float(x)], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def whole_job_mlups(world, fluid_nodes, steps, ms_max):
    """Whole-job throughput of `world` replicas that each advanced `fluid_nodes` for `steps`
    steps, timed by the slowest rank (ms_max)."""
    return world * fluid_nodes * steps / (ms_max * 1e-3) / 1e6


def barrier(world):
    if world > 1:
        import torch.distributed as dist
        dist.barrier()


def make_lattice(w, scheme, precision, kernel_path=0, graph_steps=0):
    from paper_1908_09235_gb300 import lbm
    eos = lbm.make_eos(lbm.EOS_CS, **w.eos)
    rl, rv = lbm.lbm_coexistence(eos)
    eos.rho_wall = rv
    lat = lbm.Lattice(w.nx, w.ny, w.tau, scheme, circles=w.circles, eos=eos,
                      precision=precision, kernel_path=kernel_path, graph_steps=graph_steps)
    lat.init_droplet(*w.drop, rl, rv)
    return lat, (rl, rv)


def time_variant(w, scheme, precision, steps, warmup):
    """One variant as the headline is timed: `steps` steps through lbm_step (captured graphs of
    `warmup` steps, built and run by the warm-up) between CUDA events on the library's stream;
    then the same number of steps with events around every kernel for the kernel times."""
    import torch
    gs = max(2, warmup - warmup % 2)
    lat, _ = make_lattice(w, scheme, precision, graph_steps=gs)
    lat.step(gs)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    lat.step(steps)
    e1.record()
    torch.cuda.synchronize()
    ms_total = e0.elapsed_time(e1)
    ms_step, ms_bnd, _ = lat.step_timed(steps)
    info = lat.info()
    lat.close()
    return ms_step, ms_bnd, ms_total, info


def cpu_oracle_rate(w, budget_s, max_steps, openmp=False, warmup=0):
    """The FP64 CPU oracle on the same lattice, as many steps as fit the budget: the serial
    build (one thread) or the -fopenmp build of the same source (all host cores; falls back to
    the serial build where -fopenmp does not compile), after up to `warmup` untimed steps (also
    within the budget).  Returns (MLUPS, steps, seconds, threads, warm-up steps done)."""
    import oracle as O
    if openmp:
        try:
            O.build_oracle(openmp=True)
        except Exception:  # no OpenMP runtime on this host
            openmp = False
    c = w.eos
    Tc, _ = O.cs_critical(c["a"], c["b"], c["R"])
    rl, rv = O.cs_coexistence(c["a"], c["b"], c["R"], c["T_over_Tc"] * Tc)
    s = O.OracleSim(w.nx, w.ny, w.tau, scheme=O.MOD_B, circles=w.circles, eos=O.EOS_CS, G=c["G"],
                    a=c["a"], b=c["b"], R=c["R"], T_over_Tc=c["T_over_Tc"], rho_wall=rv,
                    openmp=openmp)
    s.init_droplet(*w.drop, rl, rv)
    n_fluid = int((s.flags() & 1 == 0).sum())
    warm, t0 = 0, time.perf_counter()
    while warm < warmup and time.perf_counter() - t0 < budget_s / 2:
        s.step(1)
        warm += 1
    done, t0 = 0, time.perf_counter()
    while done < max_steps:
        s.step(1)
        done += 1
        if time.perf_counter() - t0 > budget_s:
            break
    dt = time.perf_counter() - t0
    return n_fluid * done / dt / 1e6, done, dt, O.num_threads(openmp), warm


def run_reference(args, w):
    """The oracle as the reference arm: its -fopenmp build on all host cores."""
    world, rank, _ = dist_setup()
    if rank != 0:
        return
    budget = min(150.0, max(10.0, 3.0 * args.steps))  # a bounded sample: a few minutes at most
    mlups, done, dt, cores, warm = cpu_oracle_rate(w, budget_s=budget, max_steps=args.steps,
                                                   openmp=True, warmup=args.warmup)
    line = {"impl": "reference", "metric": METRIC, "value": round(mlups, 3), "unit": UNIT,
            "n_gpus": 0, "steps": done, "warmup": warm, "ms_per_step": round(1e3 * dt / done, 3),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": {"workload": w.name, "scheme": "mod_b"},
            "cpu_baseline": {"value": round(mlups, 3), "unit": UNIT, "cores": cores,
                             "kind": "oracle",
                             "sample": "%d FP64 time steps of the %dx%d lattice (%.1f s), %s"
                                       % (done, w.nx, w.ny, dt,
                                          "OpenMP build" if cores > 1 else "serial build")},
            "e2e": {"value": round(mlups, 3), "unit": UNIT, "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def run_e2e(w, steps):
    """Same metric through the public API with host buffers: upload rho, u from pinned host memory,
    run the steps, read rho, u back; all inside the timed region (the context and its captured
    graph of steps are set up before it)."""
    import numpy as np
    import torch

    from paper_1908_09235_gb300 import lbm
    lat, (rl, rv) = make_lattice(w, lbm.MOD_B, lbm.FP32_DEV)
    n = w.nx * w.ny
    host = [torch.empty(n, dtype=torch.float64, pin_memory=True) for _ in range(3)]
    rho, ux, uy = lat.fields()  # a realistic initial state (the droplet), staged in pinned memory
    host[0].numpy()[:] = np.nan_to_num(rho.ravel(), nan=rv)
    host[1].numpy()[:] = np.nan_to_num(ux.ravel())
    host[2].numpy()[:] = np.nan_to_num(uy.ravel())
    out = [torch.empty(n, dtype=torch.float64, pin_memory=True) for _ in range(3)]
    lib = lbm.load_library()
    # one-time set-up outside the timed region: the same upload once (it fixes the automatic
    # rho_ref from this state) and the context's captured graph of steps, which stays valid
    # across lbm_init_fields while rho_ref is unchanged
    lbm._check(lat.ctx, lib.lbm_init_fields(lat.ctx, host[0].data_ptr(), host[1].data_ptr(),
                                            host[2].data_ptr()))
    lat.step(32)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    lbm._check(lat.ctx, lib.lbm_init_fields(lat.ctx, host[0].data_ptr(), host[1].data_ptr(),
                                            host[2].data_ptr()))
    t1 = time.perf_counter()  # lbm_init_fields blocks (it reads rho_ref back)
    lbm._check(lat.ctx, lib.lbm_step(lat.ctx, steps))
    lbm._check(lat.ctx, lib.lbm_fields(lat.ctx, out[0].data_ptr(), out[1].data_ptr(),
                                       out[2].data_ptr()))
    dt = time.perf_counter() - t0
    info = lat.info()
    lat.close()
    split = {"upload_and_init_ms": round(1e3 * (t1 - t0), 2),
             "steps_and_download_ms": round(1e3 * (t0 + dt - t1), 2)}
    return info["n_fluid"] * steps / dt / 1e6, 24 * n / steps, 24 * n / steps, split


# Table 1 of the paper (Sec. 4.2): 2L/D, separation angle (degrees), drag coefficient
TABLE1 = {20: {"scheme A": (1.90, 41.35, 2.130), "scheme B": (1.91, 41.56, 2.133),
               "Dennis and Chang 1970": (1.88, 43.7, 2.045)},
          40: {"scheme A": (4.61, 53.93, 1.590), "scheme B": (4.64, 53.93, 1.593),
               "Dennis and Chang 1970": (4.69, 53.8, 1.522)}}


def cylinder_wake(ux, uy, cx, cy, r, D):
    """Wake length 2L/D (L from the cylinder's rearmost point to where u_x on the centre line
    turns positive again) and separation angle (degrees from the rear stagnation point, where the
    tangential velocity changes sign on rings just outside the surface, mean of both halves,
    extrapolated linearly from the rings to the surface)."""
    import numpy as np
    j = int(round(cy))
    row = ux[j]
    x_rear = cx + r
    L = float("nan")
    for i in range(int(np.ceil(x_rear)), row.size - 1):
        if np.isfinite(row[i]) and np.isfinite(row[i + 1]) and row[i] < 0.0 <= row[i + 1]:
            L = i + row[i] / (row[i] - row[i + 1]) - x_rear
            break

    def bilinear(a, x, y):
        i0, j0 = int(np.floor(x)), int(np.floor(y))
        tx, ty = x - i0, y - j0
        return ((1 - tx) * (1 - ty) * a[j0, i0] + tx * (1 - ty) * a[j0, i0 + 1] +
                (1 - tx) * ty * a[j0 + 1, i0] + tx * ty * a[j0 + 1, i0 + 1])

    def angle_at(rs):
        angles = []
        for side in (1.0, -1.0):
            prev = None
            for k in range(1, 1800):
                th = np.radians(0.1 * k)
                x, y = cx + rs * np.cos(th), cy + side * rs * np.sin(th)
                # tangential velocity towards the front, mirrored onto the upper half (u_y is
                # odd under the reflection y -> 2 cy - y, u_x even)
                ut = -np.sin(th) * bilinear(ux, x, y) + side * np.cos(th) * bilinear(uy, x, y)
                if prev is not None and prev > 0.0 >= ut:
                    angles.append(0.1 * (k - 1) + 0.1 * prev / (prev - ut))
                    break
                prev = ut
        return float(np.mean(angles)) if len(angles) == 2 else float("nan")

    # rings from r + 1.5 (the nearest whose interpolation cells hold no solid node) outwards;
    # the angle at the surface is their linear extrapolation to radius r
    radii = np.array([1.5, 2.0, 2.5, 3.0]) + r
    th = np.array([angle_at(v) for v in radii])
    theta = float(np.polyval(np.polyfit(radii - r, th, 1), 0.0)) if np.all(np.isfinite(th)) \
        else float("nan")
    return 2.0 * L / D, theta


def run_cylinder_flow(args):
    """Steady flow past a circular cylinder, Sec. 4.2: domain 40 D x 25 D, cylinder of diameter
    D at (15 D, 12.5 D), U0 = 0.1, Zou-He velocity inlet, fully developed outlet, periodic in y,
    Re = U0 D / nu.  Runs each (Re, scheme) until the drag changes by less than 1e-6 (relative)
    over 1000 steps, then reports C_d = F_x / (0.5 rho U0^2 D), 2L/D and the separation angle
    beside Table 1 of the paper."""
    import numpy as np
    import torch

    from paper_1908_09235_gb300 import lbm
    torch.cuda.set_device(0)
    D = args.cyl_diameter
    nx, ny, U0 = 40 * D, 25 * D, 0.1
    cx, cy, r = 15.0 * D, 12.5 * D, 0.5 * D
    runs = []
    for Re in (20, 40):
        nu = U0 * D / Re
        tau = 3.0 * nu + 0.5
        for name in ("mod_a", "mod_b"):
            lat = lbm.Lattice(nx, ny, tau, lbm.SCHEMES[name], circles=[(cx, cy, r)],
                              eos=lbm.make_eos(lbm.EOS_NONE),
                              precision=lbm.PRECISIONS[args.precision])
            ux0 = np.full(nx * ny, U0)
            lat.init_fields(np.ones(nx * ny), ux0, np.zeros(nx * ny))
            lat.set_inflow(U0)
            t0 = time.perf_counter()
            cd_prev, steps, conv = None, 0, False
            while steps < args.cyl_max_steps:
                lat.step(1000)
                steps += 1000
                cd = lat.force()[0] / (0.5 * U0 * U0 * D)
                if cd_prev is not None and abs(cd - cd_prev) < 1e-6 * abs(cd):
                    conv = True
                    break
                cd_prev = cd
            wall = time.perf_counter() - t0
            rho, ux, uy = lat.fields()
            n_fluid = lat.info()["n_fluid"]
            lat.close()
            wake, theta = cylinder_wake(ux, uy, cx, cy, r, D)
            runs.append({"Re": Re, "scheme": name, "tau": round(tau, 4), "steps": steps,
                         "converged": conv, "Cd": round(cd, 4), "2L/D": round(wake, 3),
                         "theta_s_deg": round(theta, 2),
                         "mlups": round(n_fluid * steps / wall / 1e6, 1),
                         "table1": TABLE1[Re]})
    print(json.dumps({"report": "steady flow past a circular cylinder (Sec. 4.2, Table 1)",
                      "D": D, "domain": [nx, ny], "U0": U0, "storage": args.precision,
                      "runs": runs}), flush=True)


# Sec. 3.2 (Figs. 8 and 11): what the paper states about the mass of its droplet-on-cylinder run
PAPER_MASS = {"zhao_yong": "about 40% of the mass lost after 1500 steps (Fig. 8)",
              "mod_a": "maximum variation of the normalised mass about 0.01% (Fig. 11)",
              "mod_b": "maximum variation of the normalised mass about 0.01% (Fig. 11)"}


def run_paper_mass(args):
    """The paper's own two-phase test (Sec. 3.2): a 300 x 350 periodic lattice, a cylinder of
    radius 70 at (150, 130), a droplet of radius 50 on its top (tanh profile, width 5, the
    printed coexistence densities), the exponential pseudopotential with |G| = 10/3 (attractive,
    reading r1), nu = 0.15 (tau = 0.95), virtual wall density 1.5; every curved-wall scheme in
    the storage format of --precision (FP64 for the comparison with the paper), the normalised
    mass m/m0 after each chunk of steps (Figs. 8 and 11), beside what the paper states."""
    import torch

    from paper_1908_09235_gb300 import lbm
    torch.cuda.set_device(0)
    marks = (100, 500, 1000, 1500, 2000, 5000, 10000, 20000, 40000, 60000)
    marks = tuple(m for m in marks if m <= args.mass_steps)
    runs = []
    for name in ("hbb", "fh", "mls", "bouzidi_l", "bouzidi_q", "zhao_yong", "mod_a", "mod_b",
                 "bao"):
        eos = lbm.make_eos(lbm.EOS_EXP, G=-10.0 / 3.0, psi0=1.0, rho0=1.0, rho_wall=1.5)
        lat = lbm.Lattice(300, 350, 0.95, lbm.SCHEMES[name], circles=[(150.0, 130.0, 70.0)],
                          eos=eos, precision=lbm.PRECISIONS[args.precision])
        lat.init_droplet(150.0, 200.0, 50.0, 5.0, 2.783, 0.3675)
        m0 = lat.mass()
        done, curve, status, dev = 0, {}, "ok", 0.0
        t0 = time.perf_counter()
        for m in marks:
            lat.step(m - done)
            done = m
            try:
                r = lat.mass() / m0
            except lbm.LBMError as e:
                status = "unstable (status %d) before step %d" % (e.status, m)
                break
            curve[str(m)] = float("%.9f" % r)
            dev = max(dev, abs(r - 1.0))
        wall = time.perf_counter() - t0
        lat.close()
        runs.append({"scheme": name, "status": status, "mass_over_m0": curve,
                     "max_abs_mass_variation": float("%.3e" % dev),
                     "seconds": round(wall, 2), "paper": PAPER_MASS.get(name)})
    # Sec. 4.2 (Figs. 10-12): the modified schemes and Bao's at three wettabilities (virtual wall
    # densities rho_V, halfway and three quarters towards rho_L; the paper's contact angles 30,
    # 90 and 120 degrees are not tied to wall densities there), to 100000 steps
    rl, rv = 2.783, 0.3675
    wet = []
    for rw in (rv, rv + 0.5 * (rl - rv), rv + 0.75 * (rl - rv)):
        for name in ("mod_a", "mod_b", "bao"):
            eos = lbm.make_eos(lbm.EOS_EXP, G=-10.0 / 3.0, psi0=1.0, rho0=1.0, rho_wall=rw)
            lat = lbm.Lattice(300, 350, 0.95, lbm.SCHEMES[name],
                              circles=[(150.0, 130.0, 70.0)], eos=eos,
                              precision=lbm.PRECISIONS[args.precision])
            lat.init_droplet(150.0, 200.0, 50.0, 5.0, rl, rv)
            m0, dev, status = lat.mass(), 0.0, "ok"
            for _ in range(10):
                lat.step(10000)
                try:
                    dev = max(dev, abs(lat.mass() / m0 - 1.0))
                except lbm.LBMError as e:
                    status = "unstable (status %d)" % e.status
                    break
            lat.close()
            wet.append({"rho_wall": round(rw, 4), "scheme": name, "steps": 100000,
                        "status": status, "max_abs_mass_variation": float("%.3e" % dev)})
    print(json.dumps({"report": "droplet on a cylinder, mass over time (Sec. 3.2, Figs. 8, 11)",
                      "domain": [300, 350], "tau": 0.95, "storage": args.precision,
                      "runs": runs, "wettability": wet}), flush=True)


def run_paper_gravity(args):
    """The paper's single-phase leakage test (Sec. 3.1, Figs. 3-5): a 100 x 50 lattice, periodic in
    x, flat solid walls below and above with the fraction q = 0.1 .. 0.9 on both, tau = 1,
    gravity (0, -rho g) with g = 0.001, uniform rho = 1 at rest initially; the averaged mass
    change rate eps = |m - m0| / m0 x 100% after 60000 steps (Fig. 5) for each scheme, in the
    storage format of --precision (FP64 for the comparison with the paper)."""
    import numpy as np
    import torch

    from paper_1908_09235_gb300 import lbm
    torch.cuda.set_device(0)
    nx, ny = 100, 50
    qs = [n / 10 for n in range(1, 10)]
    table = {}
    for name in ("mls", "bouzidi_l", "bouzidi_q", "zhao_yong", "mod_a", "mod_b"):
        row = {}
        for q in qs:
            lat = lbm.Lattice(nx, ny, 1.0, lbm.SCHEMES[name], wall_q_lo=q, wall_q_hi=q,
                              eos=lbm.make_eos(lbm.EOS_NONE, gy=-0.001),
                              precision=lbm.PRECISIONS[args.precision])
            lat.init_fields(np.ones(nx * ny))
            m0 = lat.mass()
            lat.step(args.gravity_steps)
            try:
                row["%.1f" % q] = float("%.4g" % (abs(lat.mass() - m0) / m0 * 100.0))
            except lbm.LBMError as e:
                row["%.1f" % q] = "unstable (status %d)" % e.status
            lat.close()
        table[name] = row
    print(json.dumps({"report": "static flow under gravity, averaged mass change rate eps in % "
                                "(Sec. 3.1, Fig. 5)", "domain": [nx, ny], "tau": 1.0, "g": 0.001,
                      "steps": args.gravity_steps, "storage": args.precision, "eps": table,
                      "paper": "Zhao-Yong's eps much larger than the other schemes' at every q; "
                               "MLS and Bouzidi conserve mass at q = 0.5 only"}), flush=True)


def _field_errors(got, ref):
    import numpy as np
    m = np.isfinite(ref[0])
    if not np.array_equal(np.isfinite(got[0]), m) and not np.all(np.isfinite(got[0][m])):
        return {"finite": False}
    drho = np.abs(got[0][m] - ref[0][m])
    du = np.maximum(np.abs(got[1][m] - ref[1][m]), np.abs(got[2][m] - ref[2][m]))
    return {"finite": True,
            "rho_normwise": float("%.3e" % (drho.max() / np.max(ref[0][m]))),
            "rho_max_rel": float("%.3e" % np.max(drho / ref[0][m])),
            "rho_rms": float("%.3e" % np.sqrt(np.mean(drho ** 2))),
            "u_max_abs": float("%.3e" % du.max()),
            "u_max_ref": float("%.3e" % np.max(np.hypot(ref[1][m], ref[2][m])))}


def precision_measure(side, checkpoints, fp16_bound=1e-3):
    """The storage formats against the FP64 CPU oracle on one droplet-on-cylinder lattice of
    the given side (the 4096^2 geometry scaled: cylinder 600/4096 L, droplet 800/4096 L), scheme
    B: FP64, FP32 deviation and FP16 deviation storage on the GPU and the oracle's -fopenmp build
    on all host cores, compared after each step count in `checkpoints` (rho and u errors,
    total-mass drift).  Also the last checkpoint up to which the FP16 format's normwise rho
    error stays below fp16_bound."""
    import numpy as np
    import torch

    import oracle as O
    from paper_1908_09235_gb300 import lbm, workloads
    w = workloads.droplet_on_cylinder(side, 600.0 / 4096 * side, 800.0 / 4096 * side)
    openmp = True
    try:
        O.build_oracle(openmp=True)
    except Exception:  # no OpenMP runtime on this host: the serial build
        openmp = False
    c = w.eos
    Tc, _ = O.cs_critical(c["a"], c["b"], c["R"])
    rl, rv = O.cs_coexistence(c["a"], c["b"], c["R"], c["T_over_Tc"] * Tc)
    s = O.OracleSim(w.nx, w.ny, w.tau, scheme=O.MOD_B, circles=w.circles, eos=O.EOS_CS, G=c["G"],
                    a=c["a"], b=c["b"], R=c["R"], T_over_Tc=c["T_over_Tc"], rho_wall=rv,
                    openmp=openmp)
    s.init_droplet(*w.drop, rl, rv)
    lats, m0 = {}, {}
    for pname in ("fp64", "fp32_dev", "fp16_dev"):
        lats[pname], _ = make_lattice(w, lbm.MOD_B, lbm.PRECISIONS[pname])
        m0[pname] = lats[pname].mass()
    rows, done, oracle_s = [], 0, 0.0
    fp16_ok_until = 0
    checkpoints = sorted(int(c) for c in checkpoints)
    steps = checkpoints[-1]
    for target in checkpoints:
        n = target - done
        t0 = time.perf_counter()
        s.step(n)
        oracle_s += time.perf_counter() - t0
        ref = s.fields()
        done += n
        row = {"step": done}
        for pname, lat in lats.items():
            lat.step(n)
            try:
                drift = abs(lat.mass() / m0[pname] - 1.0)
            except lbm.LBMError:
                drift = None
            e = _field_errors(lat.fields(), ref)
            e["mass_drift"] = float("%.3e" % drift) if drift is not None else None
            row[pname] = e
        if row["fp16_dev"].get("finite") and row["fp16_dev"]["rho_normwise"] < fp16_bound and \
                fp16_ok_until == done - n:
            fp16_ok_until = done  # every earlier checkpoint was within the bound too
        rows.append(row)
    for lat in lats.values():
        lat.close()
    torch.cuda.synchronize()
    n_fluid = int((s.flags() & 1 == 0).sum())
    return {"workload": w.name, "scheme": "mod_b", "steps": steps, "checkpoints_steps": checkpoints,
            "oracle": {"build": "-fopenmp" if openmp else "serial",
                       "threads": O.num_threads(openmp), "seconds": round(oracle_s, 1),
                       "mlups": round(n_fluid * steps / oracle_s / 1e6, 2)},
            "fp16_normwise_bound": fp16_bound,
            "fp16_within_bound_through_step": fp16_ok_until,
            "checkpoints": rows}


def run_precision_report(args):
    """The reduced-precision formats on long runs (--precision-report): against the FP64 CPU
    oracle on the smallest side of --report-sides (every --report-every steps), and total-mass
    drift of the FP32 and FP16 formats on the larger sides (no oracle there: its run would take
    hours)."""
    import torch

    from paper_1908_09235_gb300 import lbm, workloads
    torch.cuda.set_device(0)
    sides = sorted(int(v) for v in args.report_sides.split(","))
    steps, every = args.report_steps, args.report_every
    marks = sorted({c for c in (10, 20, 50, 100, 200, 500, 1000, 2000, 5000, 10000) if c < steps}
                   | set(range(every, steps + 1, every)) | {steps})
    out = {"report": "reduced precision, droplet on cylinder, scheme B", "steps": steps,
           "vs_oracle": precision_measure(sides[0], marks), "drift_only": []}
    for L in sides[1:]:
        w = workloads.droplet_on_cylinder(L, 600.0 / 4096 * L, 800.0 / 4096 * L)
        for pname in ("fp32_dev", "fp16_dev"):
            lat, _ = make_lattice(w, lbm.MOD_B, lbm.PRECISIONS[pname])
            m0 = lat.mass()
            drift, done, status = [], 0, "ok"
            while done < steps:
                n = min(every, steps - done)
                lat.step(n)
                done += n
                try:
                    drift.append(abs(lat.mass() / m0 - 1.0))
                except lbm.LBMError as e:
                    status = str(e)
                    break
            lat.close()
            out["drift_only"].append({"side": L, "storage": pname, "steps": done,
                                      "status": status,
                                      "mass_drift_every_%d" % every:
                                          [float("%.3e" % d) for d in drift],
                                      "max_mass_drift": float("%.3e" % max(drift))
                                      if drift else None})
    print(json.dumps(out), flush=True)


def run_profile_case(args):
    """A single lattice of side L stepped a few times (the benchmark's 4096^2 lattice, or one of
    side L with cylinder 0.15 L and droplet 0.2 L); the case of ncu captures."""
    import torch

    from paper_1908_09235_gb300 import lbm, workloads
    L = args.profile_case
    # 4096: the benchmark's own lattice; other sides: the same shape scaled
    w = workloads.LARGE if L == workloads.LARGE.nx else workloads.droplet_on_cylinder(L, 0.15 * L,
                                                                                      0.2 * L)
    lat, _ = make_lattice(w, lbm.SCHEMES[args.scheme], lbm.PRECISIONS[args.precision],
                          args.kernel_path)
    lat.step_timed(args.warmup)
    ms = lat.step_timed(args.steps)
    torch.cuda.synchronize()
    info = lat.info()
    lat.close()
    print(json.dumps({"profile_case": w.name, "precision": args.precision, "scheme": args.scheme,
                      "kernel_path": args.kernel_path,
                      "steps": args.steps, "step_kernel_us": 1e3 * ms[0] / args.steps,
                      "boundary_kernel_us": 1e3 * ms[1] / args.steps,
                      "fluid_nodes": info["n_fluid"]}), flush=True)


SCHED_NAMES = ("strided", "claim", "claim_largest_first")


def _batch_member(lbm, w):
    eos = lbm.make_eos(lbm.EOS_CS, **w["eos"])
    rl, rv = lbm.lbm_coexistence(eos)
    eos.rho_wall = rv
    return lbm.make_domain(w["nx"], w["ny"], w["tau"], lbm.MOD_B, circles=[w["cyl"]], eos=eos,
                           droplet=tuple(w["drop"]) + (rl, rv))


def batched_measure(n_domains, precision, steps, warmup, base_count=16, accuracy_sample=4):
    """The batched workload (n_domains uneven droplet-on-cylinder lattices, sides 64..512,
    seeded) in one batch: one set of launches per time step under a CUDA graph, tile height and
    tile-queue schedule chosen by the batch's tuner; `steps` timed steps of every lattice.
    Throughput over all lattices and over the lattices that stayed finite (a diverged lattice
    costs the same per step but its result is void), beside the plain loop that advances one
    FP64 lattice at a time (the first base_count lattices, 10 steps each), and the density of
    accuracy_sample finite lattices against the same lattice run alone in FP64."""
    import numpy as np
    import torch

    from paper_1908_09235_gb300 import lbm, workloads
    ws = workloads.batched_domains(n_domains)
    prec = lbm.PRECISIONS[precision]
    b = lbm.Batch(prec, lbm.EOS_CS, max_domains=len(ws))
    slots = [b.add(_batch_member(lbm, w), 10**9) for w in ws]
    b.tune(3)
    trials = b.tune_trials()
    info = b.info()
    b.step(warmup)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    with Clocks(0) as clk:
        e0.record()
        b.step(steps)
        e1.record()
        torch.cuda.synchronize()
    ms = e0.elapsed_time(e1)
    split = b.step_timed(5)
    unstable, finite_nodes = [], 0
    for w, s_ in zip(ws, slots):
        try:
            b.mass(s_)
            finite_nodes += lbm.lbm_info(b.ctx(s_))["n_fluid"]
        except lbm.LBMError:
            unstable.append(w["name"])
    # accuracy: a few finite lattices, spread over the workload, against the same lattice run
    # alone with FP64 storage for the same number of steps
    total = warmup + steps + 5
    acc = []
    stride = max(1, len(ws) // max(1, accuracy_sample))
    for k in sorted(range(len(ws)), key=lambda i: (i % stride, i)):  # 0, s, 2s, .., then 1, s+1, ..
        if len(acc) >= accuracy_sample:
            break
        if ws[k]["name"] in unstable:
            continue
        rho_b = b.fields(slots[k])[0]
        w = ws[k]
        eos = lbm.make_eos(lbm.EOS_CS, **w["eos"])
        rl, rv = lbm.lbm_coexistence(eos)
        eos.rho_wall = rv
        lat = lbm.Lattice(w["nx"], w["ny"], w["tau"], lbm.MOD_B, circles=[w["cyl"]], eos=eos)
        lat.init_droplet(*w["drop"], rl, rv)
        lat.step(total)
        rho64 = lat.fields()[0]
        lat.close()
        m = np.isfinite(rho64)
        d = np.abs(rho_b[m] - rho64[m])
        acc.append({"lattice": w["name"], "side": w["nx"],
                    "rho_normwise": float("%.3e" % (d.max() / np.max(rho64[m])))})
    b.close()
    value = info["fluid_nodes"] * steps / (ms * 1e-3) / 1e6
    base_nodes, base_ms = 0, 0.0
    for w in ws[:base_count]:
        eos = lbm.make_eos(lbm.EOS_CS, **w["eos"])
        rl, rv = lbm.lbm_coexistence(eos)
        eos.rho_wall = rv
        lat = lbm.Lattice(w["nx"], w["ny"], w["tau"], lbm.MOD_B, circles=[w["cyl"]], eos=eos)
        lat.init_droplet(*w["drop"], rl, rv)
        lat.step_timed(2)
        _, _, t = lat.step_timed(10)
        base_nodes += lat.info()["n_fluid"] * 10
        base_ms += t
        lat.close()
    base = base_nodes / (base_ms * 1e-3) / 1e6
    return {"workload": "batched_droplets_%d" % len(ws), "storage": precision, "scheme": "mod_b",
            "steps": steps, "lattices": info["active"], "nodes": info["nodes"],
            "fluid_nodes": info["fluid_nodes"], "tiles": info["tiles"],
            "tile": [info["tile_cols"], info["tile_rows"]],
            "schedule": SCHED_NAMES[info["schedule"]], "graph": True,
            "ms_per_step": round(ms / steps, 4), "mlups": round(value, 1),
            "mlups_finite_lattices": round(finite_nodes * steps / (ms * 1e-3) / 1e6, 1),
            "unstable_lattices": len(unstable), "unstable_names": unstable,
            "tuner_ms_per_launch": {"%dx%d/%s" % (info["tile_cols"], r, SCHED_NAMES[sc]):
                                    round(t, 4) for r, sc, t in trials},
            "split_ms_per_step": {"step_kernel": round(split[1] / 5, 4),
                                  "boundary_and_advance": round(split[2] / 5, 4)},
            "plain_fp64_loop_mlups": round(base, 1),
            "speedup_vs_plain_fp64_loop": round(value / base, 2),
            "accuracy_vs_fp64_alone": {
                "lattices": len(acc), "steps": total,
                "max_rho_normwise": max((a["rho_normwise"] for a in acc), default=None),
                "samples": acc,
                "how": "finite batched lattices (this storage, in the batch) against the same "
                       "lattice run alone with FP64 storage"},
            "clocks": clk.summary()}


def run_batched(args):
    """The batched workload as its own JSON line (--batched)."""
    import torch
    torch.cuda.set_device(0)
    r = batched_measure(args.batch_domains, args.precision, args.batch_steps, args.warmup)
    line = {"metric": METRIC, "value": r["mlups"], "unit": UNIT, "n_gpus": 1,
            "steps": args.batch_steps, "warmup": args.warmup, "ms_per_step": r["ms_per_step"],
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "f64" if args.precision == "fp64" else "f32", "data": "synthetic",
            "config": {k: r[k] for k in ("workload", "storage", "scheme", "lattices", "nodes",
                                         "fluid_nodes", "tiles", "tile", "schedule", "graph")},
            "batched": r, "clocks": r["clocks"]}
    print(json.dumps(line), flush=True)


def served_measure(n, rate, steps_lo, steps_hi, slots, hbm_gb, chunk, accuracy_sample=0,
                   plain_subset=0):
    """A served stream of droplet-on-cylinder requests (Poisson arrivals, side log-uniform
    128..1024, steps uniform, scheme from the five variants) through the continuous-batching
    server with FP32 deviation storage.  Beside it:
    - the plain loop that runs one FP64 lattice at a time: modelled for the whole stream (FIFO
      queue with measured FP64 rates per size) and, for the first plain_subset arrivals, run
      for real (serve.run_one_at_a_time) next to the model's figures for the same subset;
    - accuracy: up to accuracy_sample finished stable requests (side <= 512) re-run alone in
      FP64; the served FP32 density against it."""
    import numpy as np
    import torch

    from paper_1908_09235_gb300 import lbm, serve, workloads
    reqs = workloads.served_requests(n=n, rate=rate, steps_lo=steps_lo, steps_hi=steps_hi)
    srv = serve.Server(precision=lbm.FP32_DEV, max_slots=slots,
                       hbm_bytes=int(hbm_gb * 2**30) if hbm_gb else None, chunk=chunk)
    want = [r["rid"] for r in reqs if r["nx"] <= 512][:3 * accuracy_sample]
    kept = {}

    def collect(b, slot):
        res = serve.summary_result(b, slot)
        rid = srv.slot_rid[slot]
        if rid in want and not res["unstable"] and len(kept) < accuracy_sample:
            kept[rid] = b.fields(slot)[0]
        return res

    t0 = time.perf_counter()
    with Clocks(0) as clk:
        done = srv.run(reqs, collect=collect)
    makespan = time.perf_counter() - t0
    srv.close()
    work = sum(r.fluid_nodes * r.steps for r in done)
    stable_work = sum(r.fluid_nodes * r.steps for r in done if not r.result.get("unstable"))
    stats = serve.latency_stats(done)
    unstable = sum(1 for r in done if r.result.get("unstable"))
    # the plain loop: per-size FP64 step rate and set-up time measured here
    sizes = [128, 256, 512, 1024]
    rate_by, setup = {}, {}
    for L in sizes:
        req = dict(workloads.served_requests(n=1, side_lo=L, side_hi=L)[0])
        t1 = time.perf_counter()
        lat = serve.request_lattice(req)
        lat.mass()
        setup[L] = time.perf_counter() - t1
        lat.step_timed(3)
        _, _, ms = lat.step_timed(20)
        rate_by[L] = lat.info()["n_fluid"] * 20 / (ms * 1e-3)
        lat.fields()
        lat.close()
    logs = np.log(sizes)

    def interp(d, L):
        return float(np.exp(np.interp(np.log(L), logs, np.log([d[s] for s in sizes]))))
    by_id = {r["rid"]: r for r in reqs}
    order = sorted(done, key=lambda r: r.arrival)
    service = [interp(setup, by_id[r.rid]["nx"]) + r.fluid_nodes * r.steps /
               interp(rate_by, by_id[r.rid]["nx"]) for r in order]
    arrivals = [r.arrival for r in order]
    base_lat = serve.fifo_latencies(arrivals, service)
    base_makespan = max(a + l for a, l in zip(arrivals, base_lat))
    out = {"workload": "served_droplets_%d" % len(reqs), "storage": "fp32_dev",
           "arrival_rate_per_s": rate, "steps_range": [steps_lo, steps_hi], "slots": slots,
           "chunk_steps": chunk, "hbm_budget_bytes": srv.hbm_bytes,
           "requests": len(done), "makespan_s": round(makespan, 2),
           "mlups": round(work / makespan / 1e6, 1),
           "mlups_stable_results": round(stable_work / makespan / 1e6, 1),
           "p50_latency_s": round(stats["p50_s"], 3), "p99_latency_s": round(stats["p99_s"], 3),
           "max_concurrent": srv.max_concurrent, "peak_admitted_bytes": srv.peak_bytes,
           "unstable_results": unstable, "node_steps": work,
           "plain_fp64_loop_model": {
               "mlups": round(work / base_makespan / 1e6, 1),
               "makespan_s": round(base_makespan, 1),
               "p50_latency_s": round(float(np.percentile(base_lat, 50)), 2),
               "p99_latency_s": round(float(np.percentile(base_lat, 99)), 2),
               "fp64_fluid_mlups_by_side": {str(k): round(v / 1e6, 1) for k, v in rate_by.items()},
               "how": "FIFO queue on the same arrivals with service time = measured FP64 "
                      "set-up + fluid nodes x steps / measured FP64 step rate of that size"},
           "clocks": clk.summary()}
    if plain_subset:
        sub = sorted(reqs, key=lambda r: r["arrival"])[:plain_subset]
        t1 = time.perf_counter()
        pdone = serve.run_one_at_a_time(sub)
        pspan = time.perf_counter() - t1
        plat = [r.latency for r in sorted(pdone, key=lambda r: r.arrival)]
        sub_ids = [r["rid"] for r in sub]
        k = [i for i, r in enumerate(order) if r.rid in sub_ids]
        model_sub = serve.fifo_latencies([arrivals[i] for i in k], [service[i] for i in k])
        out["plain_fp64_loop_run"] = {
            "requests": len(pdone), "first_arrivals": plain_subset,
            "makespan_s": round(pspan, 2),
            "mlups": round(sum(r.fluid_nodes * r.steps for r in pdone) / pspan / 1e6, 1),
            "p50_latency_s": round(float(np.percentile(plat, 50)), 3),
            "p99_latency_s": round(float(np.percentile(plat, 99)), 3),
            "model_p50_latency_s_same_requests": round(float(np.percentile(model_sub, 50)), 3),
            "model_p99_latency_s_same_requests": round(float(np.percentile(model_sub, 99)), 3),
            "how": "the first arrivals of the same stream served for real by one FP64 lattice "
                   "at a time (serve.run_one_at_a_time), arrivals on the wall clock"}
    if accuracy_sample:
        errs = []
        for rid, rho32 in kept.items():
            req = by_id[rid]
            lat = serve.request_lattice(req, lbm.FP64)
            lat.step(req["steps"])
            rho64 = lat.fields()[0]
            lat.close()
            m = np.isfinite(rho64)
            d = np.abs(rho32[m] - rho64[m])
            errs.append({"rid": rid, "side": req["nx"], "scheme": req["scheme"],
                         "steps": req["steps"],
                         "rho_normwise": float("%.3e" % (d.max() / np.max(rho64[m]))),
                         "rho_max_rel": float("%.3e" % np.max(d / rho64[m]))})
        out["accuracy_vs_fp64_alone"] = {
            "requests": len(errs),
            "max_rho_normwise": max((e["rho_normwise"] for e in errs), default=None),
            "max_rho_rel": max((e["rho_max_rel"] for e in errs), default=None),
            "samples": errs,
            "how": "finished stable served requests (FP32 deviations, in the mix) against the "
                   "same request run alone with FP64 storage"}
    return out


def run_serve(args):
    """The served stream as its own JSON line (--serve)."""
    import torch
    torch.cuda.set_device(0)
    r = served_measure(args.serve_requests, args.serve_rate, args.serve_steps_lo,
                       args.serve_steps_hi, args.serve_slots, args.serve_hbm_gb, args.serve_chunk,
                       accuracy_sample=args.serve_accuracy_sample,
                       plain_subset=args.serve_plain_subset)
    line = {"metric": METRIC, "value": r["mlups"], "unit": UNIT, "n_gpus": 1,
            "steps": None, "warmup": 0, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {k: r[k] for k in ("workload", "storage", "arrival_rate_per_s", "slots",
                                         "chunk_steps", "hbm_budget_bytes")},
            "served": r, "clocks": r["clocks"]}
    print(json.dumps(line), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=400)
    ap.add_argument("--warmup", type=int, default=20)
    ap.add_argument("--impl", default="gb300", choices=["gb300", "reference"])
    ap.add_argument("--variant-steps", type=int, default=60)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--profile-case", type=int, default=0,
                    help="only run a droplet-on-cylinder lattice of this side (for ncu)")
    ap.add_argument("--precision", default="fp32_dev", choices=["fp64", "fp32_dev", "fp16_dev"])
    ap.add_argument("--scheme", default="mod_b")
    ap.add_argument("--kernel-path", type=int, default=0,
                    help="profile case only: 0 fastest, 1 scalar tiles, 2 TMA-staged tiles, 3 vectorised")
    ap.add_argument("--batched", action="store_true",
                    help="the batched workload: many uneven lattices in one batch")
    ap.add_argument("--batch-domains", type=int, default=512)
    ap.add_argument("--batch-steps", type=int, default=5000,
                    help="batched workload: timed steps of every lattice")
    ap.add_argument("--paper-mass", action="store_true",
                    help="Sec. 3.2: mass over time of the paper's droplet on a cylinder, every scheme")
    ap.add_argument("--mass-steps", type=int, default=60000)
    ap.add_argument("--paper-gravity", action="store_true",
                    help="Sec. 3.1: mass change rate of static flow under gravity, every q")
    ap.add_argument("--gravity-steps", type=int, default=60000)
    ap.add_argument("--cylinder-flow", action="store_true",
                    help="Sec. 4.2: flow past a cylinder at Re 20 and 40 against Table 1")
    ap.add_argument("--cyl-diameter", type=int, default=40)
    ap.add_argument("--cyl-max-steps", type=int, default=400000)
    ap.add_argument("--precision-report", action="store_true",
                    help="FP32/FP16 deviation storage on long runs: mass drift and error vs FP64")
    ap.add_argument("--report-sides", default="2048,8192")
    ap.add_argument("--report-steps", type=int, default=20000)
    ap.add_argument("--report-every", type=int, default=2000)
    ap.add_argument("--serve", action="store_true",
                    help="the served stream through the continuous-batching server")
    ap.add_argument("--serve-requests", type=int, default=2000)
    ap.add_argument("--serve-rate", type=float, default=200.0)
    ap.add_argument("--serve-steps-lo", type=int, default=2000)
    ap.add_argument("--serve-steps-hi", type=int, default=20000)
    ap.add_argument("--serve-slots", type=int, default=256)
    ap.add_argument("--serve-chunk", type=int, default=200)
    ap.add_argument("--serve-hbm-gb", type=float, default=0.0,
                    help="memory budget of the server (0: 80%% of the free device memory)")
    ap.add_argument("--serve-accuracy-sample", type=int, default=8,
                    help="served requests re-run alone in FP64 to state the served accuracy")
    ap.add_argument("--serve-plain-subset", type=int, default=16,
                    help="first arrivals also served for real by the plain one-at-a-time loop")
    ap.add_argument("--no-next-rows", action="store_true",
                    help="default line without the batched / served / precision sub-objects")
    args = ap.parse_args()
    args.warmup = max(3, args.warmup)

    from paper_1908_09235_gb300 import workloads
    w = workloads.LARGE
    if args.impl == "reference":
        return run_reference(args, w)
    if args.profile_case:
        return run_profile_case(args)
    if args.batched:
        return run_batched(args)
    if args.serve:
        return run_serve(args)
    if args.precision_report:
        return run_precision_report(args)
    if args.cylinder_flow:
        return run_cylinder_flow(args)
    if args.paper_mass:
        return run_paper_mass(args)
    if args.paper_gravity:
        return run_paper_gravity(args)

    import torch
    world, rank, local = dist_setup()
    torch.cuda.set_device(local)
    from paper_1908_09235_gb300 import lbm
    lbm.load_library()

    # ---- headline: scheme B, FP32 deviation storage, through lbm_step (the path a user
    # takes): captured CUDA graphs of gs steps, which the warm-up builds and runs; CUDA events on
    # the library's stream around the K timed steps ----
    gs = max(2, min(32, args.warmup - args.warmup % 2))
    lat, _ = make_lattice(w, lbm.MOD_B, lbm.FP32_DEV, graph_steps=gs)
    lat.step(args.warmup)
    torch.cuda.synchronize()
    barrier(world)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    with Clocks(local) as clk:
        e0.record()
        lat.step(args.steps)
        e1.record()
        torch.cuda.synchronize()
    ms_total = e0.elapsed_time(e1)
    barrier(world)
    # the same steps with CUDA events around every kernel (no graphs): the step kernel's
    # average duration for the roofline and the wall pass's share
    ms_step, ms_bnd, _ = lat.step_timed(args.steps)
    torch.cuda.synchronize()
    info = lat.info()
    m_after = lat.mass()
    lat.close()
    ms_total = max_over_ranks(ms_total, world)
    n_fluid, n_all = info["n_fluid"], w.nx * w.ny
    value = whole_job_mlups(world, n_fluid, args.steps, ms_total)
    peak, peak_kind = measured_peaks()
    bpu = bytes_per_update("fp32_dev")
    achieved = n_fluid * bpu / (ms_step / args.steps * 1e-3) / 1e9
    traffic = captured_traffic()

    # the FP64 FMA pipe, measured (one timed launch of about half a second)
    fp64_gflops, fp64_ms = lbm.lbm_probe_fp64_fma(150000)
    fp64_ops = fp64_gflops / 2 * 1e9  # pipe operations per second

    variants = {}
    for prec in ("fp64", "fp32_dev", "fp16_dev"):
        for name in SCHEME_NAMES:
            s_ms, b_ms, t_ms, vinfo = time_variant(w, lbm.SCHEMES[name], lbm.PRECISIONS[prec],
                                                   args.variant_steps, 20)
            vb = bytes_per_update(prec)
            variants["%s/%s" % (prec, name)] = {
                "mlups": round(n_fluid * args.variant_steps / (t_ms * 1e-3) / 1e6, 1),
                "step_kernel_us": round(1e3 * s_ms / args.variant_steps, 2),
                "boundary_kernel_us": round(1e3 * b_ms / args.variant_steps, 2),
                "hbm_frac_step_kernel": round(
                    n_fluid * vb / (s_ms / args.variant_steps * 1e-3) / 1e9 / peak, 3)}
            if prec == "fp64":
                variants["%s/%s" % (prec, name)]["fp64_alu_frac_step_kernel"] = round(
                    FP64_PIPE_OPS_PER_NODE * n_fluid / (s_ms / args.variant_steps * 1e-3)
                    / fp64_ops, 3)

    # one end-to-end job through the C ABI: upload, at least 400 steps, download (a job of the
    # timed K steps alone would, at the driver's K = 20, mostly measure the two transfers)
    e2e_steps = max(args.steps, 400)
    e2e_value, h2d, d2h, e2e_split = run_e2e(w, e2e_steps)
    e2e_value = world * e2e_value

    # the next rows of the path, on one process only: the batched workload (200 steps of the
    # 512 lattices), the served stream at and below capacity (with a served-accuracy sample and
    # the plain FP64 loop run for real on the first arrivals), the storage formats against the
    # FP64 oracle at 2048^2 (1000 steps)
    nxt = {}
    if world == 1 and not args.no_next_rows:
        nxt["batched"] = batched_measure(512, "fp32_dev", 200, 20)
        nxt["served"] = served_measure(300, 200.0, 2000, 20000, 256, 0.0, 200,
                                       accuracy_sample=args.serve_accuracy_sample,
                                       plain_subset=args.serve_plain_subset)
        nxt["served_below_capacity"] = served_measure(120, 10.0, 2000, 20000, 256, 0.0, 200)
        nxt["precision"] = precision_measure(2048, (20, 50, 100, 250, 500, 1000))

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        mlups, done, dt, cores, _ = cpu_oracle_rate(w, budget_s=15.0, max_steps=50)
        cpu = {"value": round(mlups, 3), "unit": UNIT, "cores": cores, "kind": "oracle",
               "sample": "%d FP64 time steps of the %dx%d lattice, scheme B (%.1f s), serial build"
                         % (done, w.nx, w.ny, dt)}
        mlups, done, dt, cores, _ = cpu_oracle_rate(w, budget_s=15.0, max_steps=200,
                                                    openmp=True)
        cpu["all_cores"] = {"value": round(mlups, 3), "unit": UNIT, "cores": cores,
                            "kind": "oracle, -fopenmp build of the same source",
                            "sample": "%d FP64 time steps of the %dx%d lattice (%.1f s)"
                                      % (done, w.nx, w.ny, dt)}
        # the small parity case, 1000 steps: the serial oracle and the GPU (FP64, through lbm_step)
        from paper_1908_09235_gb300 import workloads
        sw = workloads.SMALL
        o_mlups, o_done, o_dt, _, _ = cpu_oracle_rate(sw, budget_s=15.0, max_steps=1000)
        slat, _ = make_lattice(sw, lbm.MOD_B, lbm.FP64)
        slat.step(32)
        torch.cuda.synchronize()
        t_s = time.perf_counter()
        slat.step(1000)
        slat.mass()  # blocks
        g_dt = time.perf_counter() - t_s
        s_fluid = slat.info()["n_fluid"]
        slat.close()
        cpu["small_case"] = {"workload": sw.name, "steps": 1000,
                             "oracle_serial_mlups": round(o_mlups, 3),
                             "oracle_steps_timed": o_done,
                             "gpu_fp64_mlups": round(s_fluid * 1000 / g_dt / 1e6, 1)}

    if rank == 0:
        line = {
            "metric": METRIC, "value": round(value, 1), "unit": UNIT, "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": round(ms_total / args.steps, 4), "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": w.name, "scheme": "mod_b", "storage": "fp32_dev",
                       "nodes": n_all, "fluid_nodes": n_fluid,
                       "boundary_links": info["n_links"],
                       "l2": "inputs larger than L2 (two 604 MB lattices)",
                       "stepping": "lbm_step, CUDA graphs of %d steps (kernel times: a second "
                                   "pass with events around every kernel)" % gs,
                       "parallelism": "replicas" if world > 1 else "single"},
            "mlups_all_nodes": round(world * n_all * args.steps / (ms_total * 1e-3) / 1e6, 1),
            "roofline": {"bound": "hbm", "achieved": round(achieved, 1), "peak": peak,
                         "unit": "GB/s", "frac": round(achieved / peak, 4),
                         "traffic": traffic, "peak_kind": peak_kind,
                         "kernel": "step_vec_kernel (fused force+collision+stream, "
                                   "16-byte population vectors, psi ring rows by TMA)",
                         "bytes_per_fluid_update": bpu},
            "step_kernel_us": round(1e3 * ms_step / args.steps, 2),
            "boundary_kernel_us": round(1e3 * ms_bnd / args.steps, 2),
            "gpu_launches": 2 * args.steps,
            "clocks": clk.summary(),
            "e2e": {"value": round(e2e_value, 1), "unit": UNIT,
                    "h2d_bytes_per_step": round(h2d, 1), "d2h_bytes_per_step": round(d2h, 1),
                    "job_steps": e2e_steps, "split": e2e_split},
            "cpu_baseline": cpu,
            "fp64_fma_peak": {"gflops": round(fp64_gflops, 1), "ms": round(fp64_ms, 2),
                              "kind": "measured (lbm_probe_fp64_fma, one timed launch)",
                              "pipe_ops_per_fp64_node_update": FP64_PIPE_OPS_PER_NODE},
            "variants": variants,
            "mass_after": m_after,
        }
        line.update(nxt)
        print(json.dumps(line), flush=True)
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
