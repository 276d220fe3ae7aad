"""Benchmark of the coarse-grid incremental pressure-projection (CGP) time step.

Workload (N = 1 GPU): the channel-with-cylinder problem, a seeded ~16k-triangle
Delaunay base mesh refined three times (~1.05M velocity triangles, ~0.53M vertices),
pressure increment two levels coarser, rotational form, Re = 20 on the cylinder
diameter (nu = 1e-3), dt = 0.002, solver tolerances 1e-8.  One "step" is one CGP
time step: momentum solve, injection, coarse Poisson solve, prolongation, velocity
correction, pressure update (all inside the library's CUDA kernels, replayed as a
CUDA graph).

Printed: one JSON line (rank 0).  ``value`` = time steps per second of the headline
form; ``e2e`` = the same through the C ABI with host buffers copied in and out every
step; ``roofline`` = the step's dominant kernel against the measured HBM copy
bandwidth; ``pcg_hbm`` = GB/s of the PCG iteration on synthetic n^2 x 2 Poisson
problems (n = 1024, 2048, 4096: 1.05M to 16.8M rows, all far beyond L2); ``cpu_baseline`` = the FP64 CPU oracle on a bounded sample.

``--impl reference`` times the FP64 CPU oracle itself on the same workload.
Under torchrun (N > 1) every rank runs an independent replica (the method has no
data-parallel exchange): value = steps of all ranks / max time over ranks.
"""

import argparse
import json
import os
import resource
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

METRIC = "CGP time steps/s at ~1M tris + PCG HBM GB/s; learned+FP32 vs plain FP64"
L2_BYTES = 129 * 1024 * 1024


def _peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


class ClockSampler:
    """nvidia-smi samples of SM clock and throttle reasons around a timed region.

    The sampler starts before the region (nvidia-smi needs a moment to start), every sample
    carries nvidia-smi's own timestamp, and the summary keeps the samples taken between
    `start()` and `stop()`; `stop()` waits (bounded) for the first sample after the region,
    and when the region is shorter than the interval, that sample stands for it."""

    Q = ("timestamp,index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
    NAMES = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]

    def __init__(self, gpu_index, interval_ms=50, cmd=None):
        self.gpu = gpu_index
        self.intervals = [interval_ms] if cmd else [interval_ms, 200]   # 200 ms if nvidia-smi refuses the first
        self.interval = interval_ms / 1000.0
        self.cmd = cmd
        self.proc = None
        self.samples = []          # (unix time, fields)
        self.t0 = self.t1 = None

    def _command(self, interval_ms):
        return self.cmd or ["nvidia-smi", "-i", str(self.gpu), "--query-gpu=" + self.Q,
                            "--format=csv,noheader,nounits", "-lms", str(interval_ms)]

    def __enter__(self):
        for ms in self.intervals:
            try:
                self.interval = ms / 1000.0
                self.proc = subprocess.Popen(self._command(ms), stdout=subprocess.PIPE, stderr=subprocess.DEVNULL,
                                             text=True)
                self.t = threading.Thread(target=self._read, daemon=True)
                self.t.start()
                self._wait(lambda: len(self.samples) > 0, 5.0)
            except Exception:
                self.proc = None
            if self.samples:
                break
            self.__exit__()
            self.proc = None
        return self

    @staticmethod
    def _parse(line):
        import datetime
        f = [x.strip() for x in line.split(",")]
        if len(f) < 10:
            return None
        try:
            ts = datetime.datetime.strptime(f[0], "%Y/%m/%d %H:%M:%S.%f").timestamp()
            float(f[2])
        except ValueError:
            return None
        return ts, f

    def _read(self):
        for line in self.proc.stdout:
            r = self._parse(line)
            if r is not None:
                self.samples.append(r)

    def _wait(self, cond, limit):
        end = time.time() + limit
        while not cond() and time.time() < end and self.proc is not None and self.proc.poll() is None:
            time.sleep(0.005)

    def start(self):
        self.t0 = time.time()

    def stop(self):
        self.t1 = time.time()
        t1 = self.t1
        self._wait(lambda: any(ts >= t1 for ts, _ in self.samples), 4 * self.interval + 1.0)

    def __exit__(self, *a):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()

    def window(self):
        """Samples of the timed region: those between start() and stop(), else the first
        one after start() (a region shorter than the sampling interval)."""
        rows = list(self.samples)
        if self.t0 is None or self.t1 is None:
            return rows
        inside = [r for r in rows if self.t0 <= r[0] <= self.t1]
        if inside:
            return inside
        after = [r for r in rows if r[0] >= self.t0]
        return after[:1]

    def summary(self):
        sm, mx, reasons = [], None, set()
        rows = self.window()
        for _, f in rows:
            try:
                sm.append(float(f[2]))
                mx = float(f[3])
            except ValueError:
                continue
            for n, v in zip(self.NAMES, f[6:10]):
                if v.lower() == "active":
                    reasons.add(n)
        out = {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": mx,
               "reasons": sorted(reasons), "samples": len(sm), "source": "nvidia-smi"}
        if self.t0 is not None and self.t1 is not None:
            out["window_ms"] = round(1000.0 * (self.t1 - self.t0), 1)
            out["interval_ms"] = round(1000.0 * self.interval)
        return out


class NvmlClockSampler:
    """SM clock and clock-event reasons read through NVML (the driver's management library,
    by ctypes) every `interval_ms` in a thread, so a timed region of ~100 ms still holds tens
    of samples.  Same interface and summary as ClockSampler; `ok` is False when NVML cannot
    be loaded or the device not found (the caller then falls back to nvidia-smi).  Only
    reads: no setting of the GPU is touched."""

    # bits of nvmlDeviceGetCurrentClocksEventReasons (NVML's public header)
    BITS = {"sw_power_cap": 0x4, "hw_slowdown": 0x8, "sw_thermal_slowdown": 0x20, "hw_thermal_slowdown": 0x40}
    CLOCK_SM = 1

    def __init__(self, device, interval_ms=5, lib=None):
        self.device = device
        self.interval = interval_ms / 1000.0
        self.lib = lib
        self.ok = False
        self.samples = []          # (unix time, sm MHz, reason bits)
        self.max_mhz = None
        self.t0 = self.t1 = None
        self._done = threading.Event()
        self._thread = None
        self._inited = False

    @staticmethod
    def _bus_id(device):
        try:
            import torch
            p = torch.cuda.get_device_properties(device)
            return "%08X:%02X:%02X.0" % (p.pci_domain_id, p.pci_bus_id, p.pci_device_id)
        except Exception:
            return None

    def __enter__(self):
        import ctypes
        try:
            nv = self.lib or ctypes.CDLL("libnvidia-ml.so.1")
            if nv.nvmlInit_v2() != 0:
                return self
            self.nv = nv
            self._inited = True
            h = ctypes.c_void_p()
            bus = self._bus_id(self.device)
            rc = nv.nvmlDeviceGetHandleByPciBusId_v2(bus.encode(), ctypes.byref(h)) if bus else 1
            if rc != 0:
                rc = nv.nvmlDeviceGetHandleByIndex_v2(ctypes.c_uint(int(self.device)), ctypes.byref(h))
            if rc != 0:
                return self
            self.h = h
            self.reasons = getattr(nv, "nvmlDeviceGetCurrentClocksEventReasons", None) or \
                nv.nvmlDeviceGetCurrentClocksThrottleReasons
            mx = ctypes.c_uint()
            if nv.nvmlDeviceGetMaxClockInfo(h, self.CLOCK_SM, ctypes.byref(mx)) == 0:
                self.max_mhz = float(mx.value)
            if self._sample() is None:
                return self
        except Exception:
            return self
        self.ok = True
        self._thread = threading.Thread(target=self._run, daemon=True)
        self._thread.start()
        return self

    def _sample(self):
        import ctypes
        c, r = ctypes.c_uint(), ctypes.c_ulonglong()
        if self.nv.nvmlDeviceGetClockInfo(self.h, self.CLOCK_SM, ctypes.byref(c)) != 0:
            return None
        if self.reasons(self.h, ctypes.byref(r)) != 0:
            return None
        s = (time.time(), float(c.value), int(r.value))
        self.samples.append(s)
        return s

    def _run(self):
        while not self._done.wait(self.interval):
            if self._sample() is None:
                break

    def start(self):
        self.t0 = time.time()

    def stop(self):
        self.t1 = time.time()
        end = self.t1 + 4 * self.interval + 0.5
        while self.ok and not any(ts >= self.t1 for ts, _, _ in self.samples) and time.time() < end:
            time.sleep(self.interval / 4)

    def __exit__(self, *a):
        self._done.set()
        if self._thread is not None:
            self._thread.join(timeout=2.0)
        if self._inited:
            self._inited = False
            try:
                self.nv.nvmlShutdown()
            except Exception:
                pass

    def window(self):
        """Samples between start() and stop(), else the first one after start()."""
        rows = list(self.samples)
        if self.t0 is None or self.t1 is None:
            return rows
        inside = [r for r in rows if self.t0 <= r[0] <= self.t1]
        return inside or [r for r in rows if r[0] >= self.t0][:1]

    def summary(self):
        rows = self.window()
        sm = [r[1] for r in rows]
        reasons = sorted({n for _, _, bits in rows for n, b in self.BITS.items() if bits & b})
        out = {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": self.max_mhz,
               "reasons": reasons, "samples": len(sm), "source": "nvml"}
        if self.t0 is not None and self.t1 is not None:
            out["window_ms"] = round(1000.0 * (self.t1 - self.t0), 1)
            out["interval_ms"] = round(1000.0 * self.interval)
        return out


class clock_sampler:
    """NVML sampling where the library loads, else nvidia-smi (ClockSampler)."""

    def __init__(self, device):
        self.device = device
        self.s = None

    def __enter__(self):
        s = NvmlClockSampler(self.device).__enter__()
        if not s.ok:
            s.__exit__()
            s = ClockSampler(self.device).__enter__()
        self.s = s
        return s

    def __exit__(self, *a):
        return self.s.__exit__(*a)


def workload_problem(name):
    from workloads import WORKLOADS
    w = WORKLOADS[name]
    return w, w.base_mesh()


def make_params(cg, w, form, use_graph=1, tol_inner=0.0, mass_mode=0):
    from paper_1812_00185_gb300.forms import workload_params
    return workload_params(w, form, use_graph=use_graph, tol_inner=tol_inner, mass_mode=mass_mode)


def train_guess(cg, w, args):
    """Train the learned-guess network on a held-out seed of the same workload (the timed
    run uses seed w.base_n).  Returns (FP32 parameter vector, info dict)."""
    from paper_1812_00185_gb300.forms import train_guess as train
    return train(w, pairs=args.train_pairs, iters=args.train_iters)


# algorithmic bytes per launch of each kernel kind (int32 indices, FP64 values);
# n rows, z = CSR entries of the level the kernel works on, t = triangles
def kernel_bytes(name, n, z, t=0):
    table = {
        # FP64 PCG, three kernels per iteration: p = z + beta p; q = A p (gathers p); update
        "pois_pupd": 24 * n, "pois_spmv": 12 * z + 4 * n + 16 * n, "pois_update": 64 * n,
        "mass_pupd": 24 * n, "mass_spmv": 12 * z + 4 * n + 16 * n, "mass_update": 64 * n,
        "corr_pupd": 48 * n, "corr_spmv": 12 * z + 4 * n + 32 * n, "corr_update": 120 * n,
        "bicg_v": 12 * z + 4 * n + 48 * n, "bicg_t": 12 * z + 4 * n + 48 * n,
        "bicg_p": 88 * n, "bicg_s": 72 * n, "bicg_x": 128 * n,
        "mom_assemble": 44 * z + 4 * n + 16 * n + 8 * n + 8 * n + 32 * n + 4 * n + 24 * t + 56 * t + 12 * t
                        + 16 * n + n,
        "mom_prep": 64 * n, "finish": 112 * n, "corr_rhs": 20 * z + 4 * n + 8 * n + n + 16 * n,
        "div": 20 * z + 4 * n + 16 * n + 8 * n,
        # injection fused with the coarse divergence (Eqs. 22-23): Cx, Cy values + columns,
        # U~ at the coarse vertices, the right-hand side and the tags
        "coarse_rhs": 20 * z + 4 * n + 16 * n + 8 * n + n,
        # FP32 inner kernels of the mixed form: 4-byte values, vectors and Jacobi diagonal
        # Chebyshev step of a mass solve: w = A d; e += d, r -= w, d' = c1 d + c2 D^-1 r
        "cheb_corr": 8 * z + 4 * n + 52 * n, "cheb_mass": 8 * z + 4 * n + 28 * n,
        "f32_bicg_v": 8 * z + 4 * n + 24 * n, "f32_bicg_t": 8 * z + 4 * n + 24 * n,
        "f32_bicg_p": 44 * n, "f32_bicg_s": 36 * n, "f32_bicg_x": 64 * n, "to_f32": 12 * z + 12 * n,
    }
    return table.get(name)


def level_of(name):
    return "coarse" if name.startswith("pois") or name in ("coarse_rhs", "phi_mean", "phi_sub") else "fine"


def run_gpu(args, rank, world):
    import torch
    from paper_1812_00185_gb300 import binding as cg

    dev = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(dev)
    stream = torch.cuda.current_stream()
    w, base = workload_problem(args.workload)
    t0 = time.time()
    mesh = cg.Mesh(base.xy, base.tri, base.tag, w.n_levels)
    torch.cuda.synchronize()
    t_mesh = time.time() - t0
    nv_f, nt_f, nnz_f = mesh.info(w.n_levels)
    nv_c, nt_c, nnz_c = mesh.info(w.n_levels - w.k)

    learned = {}
    if args.form in ("learned", "mixed_learned"):
        learned["params"], learned["info"] = train_guess(cg, w, args)
        learned["net"] = cg.cgp_mlp_create(mesh.handle, w.n_levels - w.k, 1)
        cg.cgp_mlp_set_params(learned["net"], learned["params"])

    def run_form(form, steps, warmup, timed=True):
        t0 = time.time()
        s = cg.Solver(mesh, make_params(cg, w, form, args.graph, args.tol_inner,
                                        cg.CGP_MASS_LUMPED if args.mass == "lumped" else cg.CGP_MASS_CONSISTENT))
        if form in ("learned", "mixed_learned"):
            cg.cgp_guess_set(s.handle, learned["net"])
        torch.cuda.synchronize()
        t_asm = time.time() - t0
        with clock_sampler(dev) as clk:
            s.step(warmup)
            U0, P0, t0_sim, st0, _ = s.fields()
            # state at the start of the timed region (fields and the previous increment the coarse guess uses)
            start = (U0, s.vector(cg.CGP_VEC_UPREV), P0, t0_sim, s.vector(cg.CGP_VEC_PHI_C))
            ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            if world > 1:
                torch.distributed.barrier()
            torch.cuda.synchronize()
            clk.start()
            ev0.record(stream)
            s.step(steps)
            ev1.record(stream)
            torch.cuda.synchronize()
            clk.stop()
        if world > 1:
            torch.distributed.barrier()
        ms = ev0.elapsed_time(ev1)
        U, P, t, st1, rc = s.fields()
        its = {k: (st1["sum_it_" + k] - st0["sum_it_" + k]) / steps for k in ("mom", "poisson", "corr", "mass")}
        its["poisson_outer"] = (st1["sum_outer_poisson"] - st0["sum_outer_poisson"]) / steps
        return s, {"ms": ms, "ms_per_step": ms / steps, "steps_per_s": 1000.0 * steps / ms, "iters": its,
                   "guess_used": st1["guess_used"] - st0["guess_used"],
                   "launches": st1["launches"] - st0["launches"], "status": rc,
                   "res_poisson": st1["res_poisson"], "res_mom": st1["res_mom"], "assemble_s": t_asm, "start": start,
                   "clocks": clk.summary()}

    head_form = args.form
    s, head = run_form(head_form, args.steps, args.warmup)
    ws_bytes = s.workspace.numel()
    # the plain FP64 form, for the comparison the metric names
    keys = ("steps_per_s", "ms_per_step", "iters", "status", "guess_used", "res_poisson")
    forms = {head_form: {k: head[k] for k in keys}}
    if not args.quick:
        # the coarse initial guesses side by side: previous increment (mixed), zero, learned;
        # and the on-chip solve with Jacobi alone instead of Jacobi + the subdomain correction
        for other in ("fp64", "mixed", "mixed_zero", "mixed_jacobi", "mixed_proj"):
            if other != head_form:
                s2, res = run_form(other, args.steps, args.warmup)
                forms[other] = {k: res[k] for k in keys}
                s2.close()

    # end to end through the C ABI: pinned host state in (U^n, U^{n-1}, P^n), one step, state
    # out (U^{n+1}, P^{n+1}), every step; it replays the first steps of the timed region from the
    # state they started from
    Uh = torch.empty((nv_f, 2), dtype=torch.float64, pin_memory=True)
    Uph = torch.empty((nv_f, 2), dtype=torch.float64, pin_memory=True)
    Ph = torch.empty(nv_f, dtype=torch.float64, pin_memory=True)
    U, Uprev, P, tcur, phic = head["start"]
    cg.cgp_set_vector(s.handle, cg.CGP_VEC_PHI_C, phic)
    Uh.numpy()[:] = U
    Uph.numpy()[:] = Uprev
    Ph.numpy()[:] = P
    e2e_steps = max(1, min(args.steps, 20))
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    ev0.record(stream)
    cur, prev = Uh.numpy(), Uph.numpy()
    for _ in range(e2e_steps):
        cg.cgp_set_fields(s.handle, cur, prev, Ph.numpy(), tcur, where=cg.CGP_HOST)
        cg.cgp_step(s.handle, 1)
        # the new U goes into the buffer of U^{n-1}, which this step no longer needs; the two
        # pinned buffers then swap roles (U^n becomes the next step's U^{n-1})
        _, _, tcur, _, _ = cg.cgp_get_fields(s.handle, U=prev, P=Ph.numpy(), where=cg.CGP_HOST)
        cur, prev = prev, cur
    ev1.record(stream)
    torch.cuda.synchronize()
    e2e_ms = ev0.elapsed_time(ev1) / e2e_steps
    e2e = {"value": 1000.0 / e2e_ms * world, "unit": "steps/s", "h2d_bytes_per_step": 8 * 5 * nv_f,
           "d2h_bytes_per_step": 8 * 3 * nv_f, "ms_per_step": round(e2e_ms, 4)}

    # per-kernel device times of one profiled step (events around every launch)
    prof = cg.cgp_profile_step(s.handle)
    peak, peak_kind = _peaks()
    kern = {}
    # prolongation (Eq. 24), one launch per level: phi at the coarse vertices copied, the
    # midpoint average of two parents (indices and values) at the new ones, phi written
    lv = [mesh.info(l)[0] for l in range(w.n_levels - w.k, w.n_levels + 1)]
    prolong_bytes = sum(8 * lv[i] + 16 * (lv[i + 1] - lv[i]) + 8 * lv[i + 1] for i in range(len(lv) - 1))
    kind, ctas, cl = s.coarse_info()
    its_c = max(1, s.fields()[3]["it_poisson"])          # inner iterations of the profiled step's coarse solve
    mixed_c = kind in (cg.CGP_COARSE_ONCHIP,) or ("mixed" in head_form and kind == cg.CGP_COARSE_PERSISTENT_MEM)
    for name, (cnt, tot) in prof.items():
        n, z, t = (nv_c, nnz_c, nt_c) if level_of(name) == "coarse" else (nv_f, nnz_f, nt_f)
        b = kernel_bytes(name, n, z, t)
        if name == "prolong":
            b = prolong_bytes / max(1, w.k)   # per launch (one per level)
        if name == "pois_onelaunch":
            # one-launch coarse PCG: the algorithmic bytes of its iterations (FP32 inner:
            # 8 nnz + 56 N per iteration; FP64: 12 nnz + 108 N), whether or not they leave chip
            b = its_c * ((8 * nnz_c + 56 * nv_c) if mixed_c else (12 * nnz_c + 108 * nv_c))
        avg = tot / cnt
        kern[name] = {"launches": cnt, "total_ms": round(tot, 4), "avg_us": round(1000 * avg, 2),
                      "GBps": round(b / (avg * 1e-3) / 1e9, 1) if b else None}
    traffic_tab = {}
    tr_path = os.path.join(ROOT, "profiles", "traffic.json")
    if os.path.exists(tr_path):
        try:
            traffic_tab = json.load(open(tr_path)).get(args.workload, {})
        except Exception:
            traffic_tab = {}
    # the dominant kernel (largest share of the profiled step) with its algorithmic HBM bytes,
    # against the measured copy bandwidth
    dom = max(kern, key=lambda k: kern[k]["total_ms"] if kern[k]["GBps"] is not None else -1)
    n, z, t = (nv_c, nnz_c, nt_c) if level_of(dom) == "coarse" else (nv_f, nnz_f, nt_f)
    bpl = (its_c * ((8 * nnz_c + 56 * nv_c) if mixed_c else (12 * nnz_c + 108 * nv_c)) if dom == "pois_onelaunch"
           else kernel_bytes(dom, n, z, t))
    roof_hbm = {"kernel": "k_pcg_onchip" if (dom == "pois_onelaunch" and kind == cg.CGP_COARSE_ONCHIP) else dom,
                "bound": "hbm", "achieved": kern[dom]["GBps"], "peak": peak, "unit": "GB/s",
                "frac": round(kern[dom]["GBps"] / peak, 4), "traffic": traffic_tab.get(dom),
                "bytes_per_launch": bpl, "avg_launch_us": kern[dom]["avg_us"],
                "peak_source": peak_kind + " (MEASURED_PEAKS.json hbm_gbs)"}
    if dom == "pois_onelaunch":
        roof_hbm.update({"inner_iterations": its_c, "us_per_iteration": round(kern[dom]["avg_us"] / its_c, 3)})
    roof = roof_hbm
    roof_smem = None
    # the on-chip coarse solve keeps its data in shared memory: its other roofline is the
    # shared-memory bandwidth of the cluster's SMs (a derived peak)
    top = max(kern, key=lambda k: kern[k]["total_ms"])
    if top == "pois_onelaunch" and kind == cg.CGP_COARSE_ONCHIP:
        _, _, _, stp, _ = s.fields()
        its = max(1, stp["it_poisson"])
        smem_bytes = its * (12 * nnz_c + 4 * nv_c)       # per inner iteration: entry (addr, value, z) + z store
        avg_s = kern[top]["avg_us"] * 1e-6
        sm_mhz = head["clocks"].get("sm_mhz") or 2070.0
        smem_peak = 128.0 * cl * sm_mhz * 1e6 / 1e9       # GB/s: 128 B per clock per SM
        ach = smem_bytes / avg_s / 1e9
        roof_smem = {"kernel": "k_pcg_onchip", "bound": "smem", "achieved": round(ach, 1), "peak": round(smem_peak, 1),
                "unit": "GB/s", "frac": round(ach / smem_peak, 4), "traffic": traffic_tab.get(top),
                "bytes_per_launch": smem_bytes, "avg_launch_us": kern[top]["avg_us"], "inner_iterations": its,
                "us_per_iteration": round(kern[top]["avg_us"] / its, 3), "cluster_ctas": cl,
                "peak_source": "derived: 128 B/clock/SM x %d SMs x %.0f MHz (median SM clock, timed region)"
                               % (cl, sm_mhz)}

    # the CPU baseline and the parity of the headline form: the FP64 oracle advances a bounded
    # number of steps from the state the timed region started from, and the GPU solver the
    # same steps from the same state; relative L2 of the fields after them
    cpu_base, parity = None, None
    if rank == 0 and world == 1 and not args.quick:
        cpu_base, n_o, _, o = cpu_oracle_rate(w, base, args.cpu_budget, state=head["start"])
        U0, Up0, P0, tt0, phic0 = head["start"]
        s.set_fields(U0, Up0, P0, tt0)
        cg.cgp_set_vector(s.handle, cg.CGP_VEC_PHI_C, phic0)
        s.step(n_o)
        Ug, Pg, tg, stg, rcg = s.fields()
        rel = lambda a, b: float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))
        parity = {"form": head_form, "oracle_steps": n_o, "from_t": round(float(tt0), 6),
                  "rel_l2_U": rel(Ug, o.U), "rel_l2_P": rel(Pg, o.P),
                  "bound": 1e-4 if "mixed" in head_form else 1e-6, "status": int(rcg)}

    # PCG iteration bandwidth on a synthetic Poisson problem far larger than L2
    pcg, transfer = None, None
    if not args.quick and rank == 0:
        pcg = [pcg_bandwidth(cg, torch, n, peak) for n in args.pcg_n]
        transfer = [transfer_bandwidth(cg, torch, n, peak) for n in args.pcg_n if n >= 2048]
    batch = None
    if not args.quick and args.batch > 0:
        batch = batch_throughput(cg, torch, args.batch, args.batch_steps, 3, args.batch_cluster, args.batch_threads,
                                 args.tol_inner)

    s.close()
    mesh.close()
    out = {
        "metric": METRIC, "value": round(head["steps_per_s"] * world, 3), "unit": "steps/s", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(head["ms_per_step"], 4),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "f32+f64" if "mixed" in head_form else "f64", "data": "synthetic",
        "config": {"workload": args.workload, "form": head_form, "fine_triangles": nt_f, "fine_vertices": nv_f,
                   "coarse_vertices": nv_c, "k": w.k, "chi": w.chi, "Re": w.Re, "dt": w.dt,
                   "tol": w.tol_poisson, "mass": args.mass, "parallelism": "replicas" if world > 1 else "single",
                   "l2": "working set %.2f GB > 129 MB L2 (no flush)" % (1e-9 * ws_bytes)},
        "e2e": e2e, "gpu_launches": int(head["launches"]), "clocks": head["clocks"], "roofline": roof,
        "kernels": kern, "setup_s": {"mesh": round(t_mesh, 3), "assemble": round(head["assemble_s"], 3)},
        "pcg_hbm": pcg, "transfer_hbm": transfer, "batch": batch, "roofline_smem": roof_smem, "forms": forms,
    }
    # the metric's comparison, decomposed: plain FP64 (Jacobi coarse PCG), then FP32 inner /
    # FP64 outer with Jacobi, + the subdomain coarse correction, + the projection guess,
    # + the learned network (the headline form)
    sps = {k: v["steps_per_s"] for k, v in forms.items()}
    if "fp64" in sps:
        out["vs_fp64"] = {k: round(sps[k], 1) for k in ("fp64", "mixed_jacobi", "mixed", "mixed_zero", "mixed_proj",
                                                        "mixed_learned") if k in sps}
        out["vs_fp64"]["headline_over_fp64"] = round(sps[head_form] / sps["fp64"], 3)
    if learned:
        out["learned"] = learned["info"]
        cg.cgp_mlp_destroy(learned["net"])
    # last, so that a reader of the line's tail sees them
    if cpu_base is not None:
        out["parity"] = parity
        out["cpu_baseline"] = cpu_base
    return out, (w, base)


def mlp_forward_time(cg, torch, w, reps=50):
    """Event-timed forward pass of the learned initial guess's MLP on the workload's Poisson
    level (batch 1, seeded inputs, the untrained initial weights)."""
    from paper_1812_00185_gb300 import learned
    base = w.base_mesh()
    mesh = cg.Mesh(base.xy, base.tri, base.tag, w.n_levels)
    lvl = w.n_levels - w.k   # the Poisson (coarse) level
    n = cg.cgp_mesh_level_info(mesh.handle, lvl)[0]
    net = cg.cgp_mlp_create(mesh.handle, lvl, 1)
    cg.cgp_mlp_set_params(net, learned.init_params(0))
    g = torch.Generator().manual_seed(0)
    r = torch.randn(n, dtype=torch.float64, generator=g).cuda()
    q = torch.randn(n, dtype=torch.float64, generator=g).cuda()
    pred = torch.empty(n, dtype=torch.float64, device="cuda")
    for _ in range(3):
        cg.cgp_mlp_forward(net, r, q, 1, pred)
    torch.cuda.synchronize()
    st = torch.cuda.current_stream()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(st)
    for _ in range(reps):
        cg.cgp_mlp_forward(net, r, q, 1, pred)
    e1.record(st)
    torch.cuda.synchronize()
    us = 1000.0 * e0.elapsed_time(e1) / reps
    cg.cgp_mlp_destroy(net)
    mesh.close()
    return {"metric": "MLP forward time", "value": round(us, 2), "unit": "us", "higher_is_better": False,
            "vertices": int(n), "batch": 1, "reps": reps, "config": {"workload": w.name, "level": lvl}}


def pcg_bandwidth(cg, torch, n_side, peak):
    """GB/s of the coarse-Poisson PCG iteration on an n_side^2 x 2 structured mesh (k = 0)."""
    from workloads import square_mesh, PHI_ZERO
    lv = 0
    nb = n_side
    while nb > 256:
        nb //= 2
        lv += 1
    base = square_mesh(nb, boundary_flags=PHI_ZERO)
    mesh = cg.Mesh(base.xy, base.tri, base.tag, lv)
    # the two-kernels-per-iteration PCG: the bandwidth-oriented path for coarse meshes far beyond L2
    prm = cg.make_params(1.0, 1.0, k=0, tol_poisson=1e-30, max_it_poisson=200, guess=cg.CGP_GUESS_ZERO,
                         bc_kind=cg.CGP_BC_CAVITY, coarse_mode=cg.CGP_COARSE_KERNELS, max_it_mom=20,
                         max_it_mass=20)
    s = cg.Solver(mesh, prm)
    nf, nc, zf, zc = cg.cgp_solver_info(s.handle)
    rhs = np.random.default_rng(0).standard_normal(nc)
    cg.cgp_poisson_solve(s.handle, rhs)          # warm-up
    prof = None
    t0 = time.time()
    phi, it, rc = cg.cgp_poisson_solve(s.handle, rhs)
    wall = time.time() - t0
    # per-kernel times come from a profiled step of this solver; a seeded random velocity
    # field gives its Poisson problem a nonzero right-hand side, so all 200 iterations run
    rng = np.random.default_rng(1)
    U = rng.standard_normal((nf, 2))
    cg.cgp_set_fields(s.handle, U, U, np.zeros(nf), 0.0)
    prof = cg.cgp_profile_step(s.handle)
    sp, up, pu = prof.get("pois_spmv"), prof.get("pois_update"), prof.get("pois_pupd")
    out = {"n": nc, "nnz": zc, "iters": it, "wall_ms_per_iter": round(1000 * wall / max(it, 1), 4)}
    if sp and up and pu:
        b_iter = kernel_bytes("pois_spmv", nc, zc) + kernel_bytes("pois_update", nc, zc) + kernel_bytes("pois_pupd", nc, zc)
        t_iter = (sp[1] / sp[0] + up[1] / up[0] + pu[1] / pu[0]) * 1e-3
        out.update({"bytes_per_iter": b_iter, "us_per_iter": round(1e6 * t_iter, 2),
                    "GBps": round(b_iter / t_iter / 1e9, 1), "frac": round(b_iter / t_iter / 1e9 / peak, 4),
                    "spmv_GBps": round(kernel_bytes("pois_spmv", nc, zc) / (sp[1] / sp[0] * 1e-3) / 1e9, 1),
                    "update_GBps": round(kernel_bytes("pois_update", nc, zc) / (up[1] / up[0] * 1e-3) / 1e9, 1),
                    "pupd_GBps": round(kernel_bytes("pois_pupd", nc, zc) / (pu[1] / pu[0] * 1e-3) / 1e9, 1)})
    s.close()
    mesh.close()
    return out


def transfer_bandwidth(cg, torch, n_side, peak):
    """GB/s of the grid-transfer kernels (Eqs. 22-24) on an n_side^2 x 2 cavity mesh with the
    pressure one level coarser (working sets far beyond L2): one profiled step (CUDA events
    around every launch); the coarse solve is cut short (tolerance 1e-2), since only the
    transfers are timed.  Algorithmic bytes: prolongation 8 N_c + 16 (N_f - N_c) + 8 N_f
    (Eq. 24, one level); injection + coarse right-hand side 20 z_c + 29 N_c (Eqs. 22-23:
    Cx, Cy values and columns, U~ at the coarse vertices, the right-hand side, the tags)."""
    from workloads import square_mesh
    lv, nb = 1, n_side // 2
    while nb > 256:
        nb //= 2
        lv += 1
    base = square_mesh(nb)
    mesh = cg.Mesh(base.xy, base.tri, base.tag, lv)
    prm = cg.make_params(400.0, 0.002, chi=0, k=1, tol_mom=1e-6, tol_poisson=1e-2, tol_mass=1e-6,
                         max_it_mom=50, max_it_poisson=50, max_it_mass=50, coarse_mode=cg.CGP_COARSE_PERSISTENT_MEM)
    s = cg.Solver(mesh, prm)
    nf, nc, zf, zc = cg.cgp_solver_info(s.handle)
    s.step(1)
    prof = cg.cgp_profile_step(s.handle)
    out = {"fine_vertices": nf, "coarse_vertices": nc}
    for name, b in (("prolong", 8 * nc + 16 * (nf - nc) + 8 * nf), ("coarse_rhs", 20 * zc + 29 * nc)):
        if name in prof:
            cnt, tot = prof[name]
            us = 1000.0 * tot / cnt
            out[name] = {"bytes": b, "us": round(us, 2), "GBps": round(b / (us * 1e-6) / 1e9, 1),
                         "frac": round(b / (us * 1e-6) / 1e9 / peak, 4)}
    s.close()
    mesh.close()
    return out


def batch_throughput(cg, torch, n_inst, steps, warmup, cluster_size=0, threads=0, tol_inner=0.0):
    """The batched form: the first n_inst of the 256 seeded uneven lid-driven cavities (sizes
    32^2..256^2 x 2 triangles, Re in [10, 400], 1-3 coarsening levels, dt = 0.005, rotational
    form, mixed precision), advanced by the library's batched step (by default one persistent
    clustered launch per step, its cluster shape autotuned unless cluster_size / threads fix
    it)."""
    from workloads import batch_instances, square_mesh
    specs = batch_instances(256)[:n_inst] if n_inst <= 256 else batch_instances(n_inst)
    specs_sorted = specs
    t0 = time.time()
    meshes, solvers = [], []
    nf_tot = nc_tot = 0
    for sp in specs:
        base = square_mesh(sp["n_fine"] >> sp["k"])
        m = cg.Mesh(base.xy, base.tri, base.tag, sp["k"])
        prm = cg.make_params(sp["Re"], 0.005, chi=1, k=sp["k"], tol_mom=1e-8, tol_poisson=1e-8, tol_mass=1e-10,
                             precision=cg.CGP_MIXED, bc_kind=cg.CGP_BC_CAVITY, tol_inner=tol_inner)
        s = cg.Solver(m, prm)
        meshes.append(m)
        solvers.append(s)
        nf_tot += s.nf
        nc_tot += s.nc
    torch.cuda.synchronize()
    t_setup = time.time() - t0
    t0 = time.time()
    b = cg.cgp_batch_create(solvers, cluster_size=cluster_size, threads=threads)
    info = cg.cgp_batch_info(b)
    mode = "whole step" if cg.cgp_batch_mode(b) == cg.CGP_BATCH_WHOLE_STEP else "graph branches"
    t_tune = time.time() - t0
    every = tuple(range(-7, 0))   # statuses are reported, not raised
    cg.cgp_batch_step(b, warmup)
    torch.cuda.synchronize()
    st_before = [cg.cgp_get_fields(s.handle, allow=every)[3] for s in solvers]
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    ev0.record()
    cg.cgp_batch_step(b, steps)
    ev1.record()
    torch.cuda.synchronize()
    ms = ev0.elapsed_time(ev1) / steps
    fields = [cg.cgp_get_fields(s.handle, allow=every) for s in solvers]
    its = [f[3] for f in fields]
    bad = [{"instance": i, "status": st["status"], **specs_sorted[i]} for i, st in enumerate(its) if st["status"] != 0]
    # the lid moves at 1: larger velocities mean the instance is diverging (the method's
    # instability on the cavity with a coarsened pressure, oracle and GPU alike)
    umax = [float(np.abs(f[0]).max()) for f in fields]
    # aggregate algorithmic HBM bytes of the timed steps, from the per-kernel models above
    # (BiCGStab iteration 24 z + 392 n; assembly 44 z + 364 n; coarse FP32-inner PCG iteration
    # 8 z_c + 56 n_c; Chebyshev step 12 z + 96 n (two components) / 12 z + 48 n (one);
    # right-hand sides, prolongation and the update 40 z + 150 n), per instance and step
    tot_bytes = 0.0
    for s, st0, st1 in zip(solvers, st_before, its):
        nf, nc, zf, zc = cg.cgp_solver_info(s.handle)
        per = lambda k: (st1["sum_it_" + k] - st0["sum_it_" + k])
        tot_bytes += per("mom") * (24 * zf + 392 * nf) + per("poisson") * (8 * zc + 56 * nc)
        tot_bytes += per("corr") * (12 * zf + 96 * nf) + per("mass") * (12 * zf + 48 * nf)
        tot_bytes += (st1["steps"] - st0["steps"]) * (84 * zf + 514 * nf)
    peak, _ = _peaks()
    gbps = tot_bytes / (ms * steps * 1e-3) / 1e9
    out = {"instances": n_inst, "form": mode, "fine_vertices": nf_tot, "coarse_vertices": nc_tot, "steps": steps,
           "ms_per_batch_step": round(ms, 4), "instance_steps_per_s": round(1000.0 * n_inst / ms, 1),
           "fine_vertex_steps_per_s": round(1000.0 * nf_tot / ms, 1), "autotune": info,
           "roofline": {"bound": "hbm", "achieved": round(gbps, 1), "peak": peak, "unit": "GB/s",
                        "frac": round(gbps / peak, 4), "bytes_per_batch_step": round(tot_bytes / steps)},
           "setup_s": round(t_setup, 2), "tune_and_capture_s": round(t_tune, 2),
           "instances_with_a_failed_solve": len(bad), "failed": bad[:16],
           "instances_with_max_velocity_above_1.5": sum(1 for u in umax if not u <= 1.5)}
    cg.cgp_batch_destroy(b)
    for s in solvers:
        s.close()
    for m in meshes:
        m.close()
    return out


def _fe_errors(cg, mesh, s, level, U, P, Ue, Pe):
    """FE L2 (sqrt(e^T M e), M the library's P1 mass matrix of the fine level) and nodal max
    errors of U and of P (P with its M-weighted mean removed, as in the paper's tables)."""
    import scipy.sparse as sp
    lev = mesh.level(level)
    M = sp.csr_matrix((s.matrix(cg.CGP_MAT_M), lev["col"], lev["rowptr"]))
    m = np.asarray(M.sum(axis=1)).ravel()
    eU = U - Ue
    eP = (P - m @ P / m.sum()) - (Pe - m @ Pe / m.sum())
    l2U = float(np.sqrt(sum(eU[:, d] @ (M @ eU[:, d]) for d in range(2))))
    return {"l2_u": l2U, "linf_u": float(np.sqrt((eU ** 2).sum(1)).max()),
            "l2_p": float(np.sqrt(eP @ (M @ eP))), "linf_p": float(np.abs(eP).max())}


def manufactured_run(cg, torch, base, n_levels, k, Re, dt, chi, bc, steps, form="fp64", mass_mode=0, tol=1e-10):
    """Advance a manufactured problem (closed-form solution) `steps` steps on the GPU;
    returns device ms per step and the errors at the final time."""
    mesh = cg.Mesh(base.xy, base.tri, base.tag, n_levels)
    prm = cg.make_params(Re, dt, chi=chi, k=k, tol_mom=tol, tol_poisson=tol, tol_mass=min(tol, 1e-10) * 1e-2,
                         max_it_mom=2000, max_it_poisson=50000, max_it_mass=2000,
                         precision=cg.CGP_MIXED if form.startswith("mixed") else cg.CGP_FP64,
                         guess=cg.CGP_GUESS_PROJ if form.endswith("proj") else cg.CGP_GUESS_PREV,
                         bc_kind=bc, mass_mode=mass_mode)
    s = cg.Solver(mesh, prm)
    st = torch.cuda.current_stream()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    e0.record(st)
    s.step(steps)
    e1.record(st)
    torch.cuda.synchronize()
    U, P, t, stats, rc = s.fields()
    Ue, Pe = cg.cgp_exact_fields(s.handle, t)
    out = {"ms_per_step": round(e0.elapsed_time(e1) / steps, 4), "t": round(t, 6), "status": int(rc),
           "fine_triangles": mesh.info(n_levels)[1], "poisson_triangles": mesh.info(n_levels - k)[1]}
    out.update({key: float("%.4e" % v) for key, v in _fe_errors(cg, mesh, s, n_levels, U, P, Ue, Pe).items()})
    s.close()
    mesh.close()
    return out


def e1_grid(cg, torch, steps=800, form="fp64"):
    """The paper's first experiment (Section 3.1, Tables 1-4): the decaying Taylor-Green vortex
    (Eqs. 28-30) at Re = 10, dt = 0.00125, to t = 1 (800 steps), on meshes of 1024 * 4^j
    triangles (four per square), the pressure increment on 1024 * 4^(j-k) triangles, standard
    (chi = 0) and rotational (chi = 1) forms.  Errors at t = 1 and the device time of each run;
    speedup = time(k = 0) / time(k) on the same fine mesh, as Table 4 defines it."""
    from workloads import crisscross_mesh
    base = crisscross_mesh(16)
    rows = []
    for j in range(4):
        for chi in (0, 1):
            t0 = None
            for k in range(j + 1):
                r = manufactured_run(cg, torch, base, j, k, 10.0, 0.00125, chi, cg.CGP_BC_TG, steps, form)
                t0 = r["ms_per_step"] if k == 0 else t0
                r.update({"M:N": "%d:%d" % (r["fine_triangles"], r["poisson_triangles"]), "chi": chi, "k": k,
                          "speedup": round(t0 / r["ms_per_step"], 3)})
                rows.append(r)
    return rows


def jobelin_tables(cg, torch, steps=100):
    """The paper's Sections 3.2-3.3 (Tables 5 and 7) on the GPU: the open-boundary vortex on
    [0,1]^2 (1024 * 4^j triangles, four per square; standard form, the paper's SCGP) and the
    vortex on the disk (unstructured, 2304 * 4^j triangles as in Fig. 1; rotational form, the
    paper's RCGP), Re = 10, dt = 0.01, to t = 1; errors at t = 1, device time per step and
    speedup = time(k = 0) / time(k) on the same fine mesh."""
    from workloads import open_square_mesh, disk_mesh
    rows = []
    cases = [("open", open_square_mesh(16), cg.CGP_BC_JOBELIN_OPEN, 0, [(2, (0, 1, 2)), (1, (0, 1)), (0, (0,))]),
             ("disk", disk_mesh(), cg.CGP_BC_JOBELIN_DISK, 1, [(2, (0, 1, 2)), (1, (0, 1))])]
    for name, base, bc, chi, grid in cases:
        for lv, ks in grid:
            t0 = None
            for k in ks:
                r = manufactured_run(cg, torch, base, lv, k, 10.0, 0.01, chi, bc, steps)
                t0 = r["ms_per_step"] if k == 0 else t0
                r.update({"vortex": name, "M:N": "%d:%d" % (r["fine_triangles"], r["poisson_triangles"]),
                          "chi": chi, "k": k, "speedup": round(t0 / r["ms_per_step"], 3)})
                rows.append(r)
    return rows


def c5_study(cg, torch, total_pairs=20000, train_iters=4000, eval_steps=200, eval_seeds=(100, 101, 102, 103)):
    """The learned initial guess trained and judged as the fifth workload states: 20,000
    (rhs, guess, increment) triples recorded by the solver (mixed form, projection guess) on
    the channel with seeds 0-7 (80 %) and on the 512^2 cavity with the pressure 1-3 levels
    coarser (20 %), one network trained across all of those meshes (Adam, batch 8), then the
    channel with the held-out seeds 100-103: coarse iterations per step and steps/s over
    `eval_steps` steps (after 5) for the zero, previous-increment, projection and learned
    guesses, the coarse solve's device time from one profiled step, and how far the learned
    form's final fields are from the projection form's (both stop at the same residual)."""
    from workloads import WORKLOADS, channel_cylinder_mesh
    from paper_1812_00185_gb300.forms import workload_params
    from paper_1812_00185_gb300.learned import PairStore, MultiMeshTrainer, init_params
    ch = WORKLOADS["channel1m_k2"]
    h = ch.extra.get("h", 0.0084)
    per_ch = int(0.8 * total_pairs) // 8
    per_cav = (total_pairs - 8 * per_ch) // 3
    sources = [(ch, channel_cylinder_mesh(seed=s, h=h), per_ch, "channel seed %d" % s) for s in range(8)]
    sources += [(WORKLOADS["cavity512_k%d" % k], None, per_cav, "cavity512 k=%d" % k) for k in (1, 2, 3)]
    t0 = time.time()
    trainer = MultiMeshTrainer(init_params(0), batch=8)
    meshes, stores, rec_info = [], [], []
    for w, base, n, label in sources:
        base = base if base is not None else w.base_mesh()
        mesh = cg.Mesh(base.xy, base.tri, base.tag, w.n_levels)
        rec = cg.Solver(mesh, workload_params(w, "mixed_proj"))
        store = PairStore(rec.nc, n)
        store.record(rec, n)
        rec.close()
        trainer.add(mesh.handle, w.n_levels - w.k, store)
        meshes.append(mesh)
        stores.append(store)
        rec_info.append({"source": label, "pairs": n, "coarse_vertices": rec.nc})
    torch.cuda.synchronize()
    t_rec = time.time() - t0
    t0 = time.time()
    hist = trainer.train(train_iters, lr=1e-3, log_every=max(1, train_iters // 8))
    torch.cuda.synchronize()
    t_train = time.time() - t0
    params = trainer.get_params()
    trainer.close()
    del stores
    for m in meshes:
        m.close()
    torch.cuda.empty_cache()
    evals = []
    for seed in eval_seeds:
        base = channel_cylinder_mesh(seed=seed, h=h)
        mesh = cg.Mesh(base.xy, base.tri, base.tag, ch.n_levels)
        net = cg.cgp_mlp_create(mesh.handle, ch.n_levels - ch.k, 1)
        cg.cgp_mlp_set_params(net, params)
        row = {"seed": seed}
        fields = {}
        for form in ("mixed_zero", "mixed", "mixed_proj", "mixed_learned"):
            s = cg.Solver(mesh, workload_params(ch, form))
            if form == "mixed_learned":
                cg.cgp_guess_set(s.handle, net)
            s.step(5)
            st0 = s.fields()[3]
            st = torch.cuda.current_stream()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            torch.cuda.synchronize()
            e0.record(st)
            s.step(eval_steps)
            e1.record(st)
            torch.cuda.synchronize()
            U, P, t, st1, rc = s.fields()
            prof = cg.cgp_profile_step(s.handle)
            pois = prof.get("pois_onelaunch")
            row[form] = {"steps_per_s": round(1000.0 * eval_steps / e0.elapsed_time(e1), 1),
                         "coarse_iters_per_step": round((st1["sum_it_poisson"] - st0["sum_it_poisson"]) / eval_steps, 2),
                         "coarse_solve_us": round(1000.0 * pois[1] / pois[0], 1) if pois else None,
                         "status": int(rc)}
            if form == "mixed_learned":
                mlp = prof.get("mlp_forward")
                row[form]["network_us"] = round(1000.0 * mlp[1] / mlp[0], 1) if mlp else None
            fields[form] = (U, P)
            s.close()
        Uj, Pj = fields["mixed_proj"]
        Ul, Pl = fields["mixed_learned"]
        row["learned_vs_proj_rel_l2"] = [float(np.linalg.norm(Ul - Uj) / np.linalg.norm(Uj)),
                                         float(np.linalg.norm(Pl - Pj) / np.linalg.norm(Pj))]
        evals.append(row)
        cg.cgp_mlp_destroy(net)
        mesh.close()
    return {"metric": "learned initial guess: training on the solver's own pairs, held-out evaluation",
            "pairs": sum(r["pairs"] for r in rec_info), "record_s": round(t_rec, 1), "train_iters": train_iters,
            "train_s": round(t_train, 1), "loss": [(int(i), int(k), round(float(l), 5)) for i, k, l in hist],
            "sources": rec_info, "eval_steps": eval_steps, "eval": evals}


def lumped_accuracy(cg, torch, steps=200):
    """Eq. 27 against Eq. 20: the rotational update with the lumped mass matrix (and the
    lumped velocity correction) against the consistent one, on the periodic-forced
    Taylor-Green vortex of the 512^2 workload (Re = 100, dt = 0.002, to t = 0.4), pressure
    1-3 levels coarser; errors against the closed form and device time per step."""
    from workloads import WORKLOADS
    rows = []
    for k in (1, 2, 3):
        w = WORKLOADS["tgp512_k2"]
        base = w.base_mesh()
        for form in ("fp64", "mixed"):
            for mass in (0, 1):
                r = manufactured_run(cg, torch, base, w.n_levels, k, w.Re, w.dt, 1, w.bc, steps, form, mass, tol=1e-8)
                r.update({"k": k, "form": form, "mass": "lumped (Eq. 27)" if mass else "consistent (Eq. 20)"})
                rows.append(r)
    return rows


def cpu_oracle_rate(w, base, budget_s, state=None):
    """Steps/s of the FP64 oracle (setup excluded), bounded to about budget_s seconds; from
    rest, or from `state` = (U, U_prev, P, t) when given.  Returns (baseline dict, steps,
    seconds, the oracle after its steps)."""
    from oracle.cgp import CGPOracle
    t0 = time.time()
    o = CGPOracle(base, w.n_levels, w.k, w.Re, w.dt, w.chi, w.bc, bc_param=w.bc_param)
    if state is not None:
        o.set_state(*state[:4])
    setup = time.time() - t0
    r0 = resource.getrusage(resource.RUSAGE_SELF)
    t0 = time.time()
    n = 0
    while True:
        o.step()
        n += 1
        if time.time() - t0 > budget_s or n >= 50:
            break
    wall = time.time() - t0
    r1 = resource.getrusage(resource.RUSAGE_SELF)
    cpu = (r1.ru_utime - r0.ru_utime) + (r1.ru_stime - r0.ru_stime)
    where = "from rest" if state is None else "from the GPU state at t = %.4g" % state[3]
    return {"value": round(n / wall, 5), "unit": "steps/s", "cores": max(1, int(round(cpu / wall))),
            "kind": "oracle", "sample": "%d oracle time steps of %s (%d fine vertices, %s) after %.1f s of setup"
                                        % (n, w.name, o.fine.n_vert, where, setup)}, n, wall, o


def aggregate_ranks(out, world, device):
    """Replicas on `world` ranks: the slowest rank's step time (device-timed and end to
    end) sets the job's time, and the job's throughput is the steps of all ranks over it.
    Every rank calls this (an all-reduce over the default process group)."""
    import torch
    import torch.distributed as dist
    t = torch.tensor([out["ms_per_step"], out["e2e"]["ms_per_step"]], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    out["ms_per_step"] = round(float(t[0].item()), 4)
    out["value"] = round(1000.0 * world / out["ms_per_step"], 3)
    out["e2e"]["ms_per_step"] = round(float(t[1].item()), 4)
    out["e2e"]["value"] = round(1000.0 * world / out["e2e"]["ms_per_step"], 3)
    return out


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=50)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="gpu", choices=["gpu", "reference"])
    ap.add_argument("--workload", default="channel1m_k2")
    ap.add_argument("--form", default="mixed_learned",
                    choices=["fp64", "mixed", "learned", "mixed_learned", "mixed_zero", "mixed_jacobi", "mixed_proj",
                             "fp64_proj"])
    ap.add_argument("--batch", type=int, default=256,
                    help="instances of the batched form (the first of the 256 seeded ones; 0: skip)")
    ap.add_argument("--batch-only", action="store_true",
                    help="print only the batched-form measurement (--batch instances, --batch-steps timed "
                         "steps after --warmup)")
    ap.add_argument("--batch-cluster", type=int, default=0, help="batched form: cluster size (0: autotuned)")
    ap.add_argument("--batch-threads", type=int, default=0, help="batched form: threads per CTA (0: autotuned)")
    ap.add_argument("--batch-steps", type=int, default=10,
                    help="timed batched steps (the cavity instances of the batch diverge within 100 steps, "
                         "in the oracle too: see the design notes)")
    ap.add_argument("--train-pairs", type=int, default=150)
    ap.add_argument("--train-iters", type=int, default=400)
    ap.add_argument("--pcg-n", type=int, nargs="+", default=[1024, 2048, 4096],
                    help="sides of the structured Poisson problems of the PCG bandwidth sweep")
    ap.add_argument("--cpu-budget", type=float, default=15.0)
    ap.add_argument("--tol-inner", type=float, default=0.0,
                    help="mixed form: residual reduction of each FP32 inner solve (0: library default)")
    ap.add_argument("--quick", action="store_true", help="skip the secondary measurements")
    ap.add_argument("--graph", type=int, default=1, choices=[0, 1],
                    help="1: replay steps as CUDA graphs; 0: eager launches (what ncu can profile)")
    ap.add_argument("--mass", default="consistent", choices=["consistent", "lumped"],
                    help="mass matrix of Eqs. 25-26 (lumped = Eq. 27)")
    ap.add_argument("--mlp-only", action="store_true",
                    help="print only the MLP forward time of the learned guess on the workload's Poisson "
                         "level (--steps forward passes)")
    ap.add_argument("--pcg-only", action="store_true",
                    help="print only the PCG bandwidth sweep (one JSON line per problem size), and the "
                         "transfer kernels' bandwidth for sizes from 2048^2")
    ap.add_argument("--e1", action="store_true",
                    help="print only the paper's Taylor-Green study (Tables 1-4) run on the GPU, one JSON line")
    ap.add_argument("--accuracy", action="store_true",
                    help="print only the Eq. 27 (lumped) against Eq. 20 (consistent) accuracy comparison")
    ap.add_argument("--jobelin", action="store_true",
                    help="print only the paper's Jobelin vortex studies (Tables 5 and 7) run on the GPU")
    ap.add_argument("--c5", action="store_true",
                    help="print only the learned-guess study: 20k recorded pairs, training, held-out seeds")
    args = ap.parse_args()
    if args.warmup < 3 and args.impl == "gpu":
        args.warmup = 3
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))

    if args.impl == "reference":
        if rank != 0:
            return 0
        w, base = workload_problem(args.workload)
        res, n, wall, _ = cpu_oracle_rate(w, base, min(120.0, 20.0 * max(1, args.steps) / 10.0))
        print(json.dumps({
            "metric": METRIC, "value": res["value"], "unit": "steps/s", "n_gpus": args.gpus, "steps": n,
            "warmup": 0, "ms_per_step": round(1000 * wall / n, 3), "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic", "impl": "reference",
            "config": {"workload": args.workload, "form": "fp64 oracle (sparse direct solves)"},
            "cpu_baseline": res,
            "e2e": {"value": res["value"], "unit": "steps/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
        }))
        return 0

    if args.mlp_only:
        if rank != 0:
            return 0
        import torch
        from paper_1812_00185_gb300 import binding as cg
        w, _ = workload_problem(args.workload)
        print(json.dumps(mlp_forward_time(cg, torch, w, args.steps)), flush=True)
        return 0
    if args.e1 or args.accuracy or args.jobelin or args.c5:
        if rank != 0:
            return 0
        import torch
        from paper_1812_00185_gb300 import binding as cg
        if args.e1:
            print(json.dumps({"metric": "Taylor-Green errors and CGP speedup (paper Section 3.1)", "form": args.form
                              if args.form in ("fp64", "mixed") else "fp64",
                              "rows": e1_grid(cg, torch, form=args.form if args.form in ("fp64", "mixed") else "fp64")}),
                  flush=True)
        if args.accuracy:
            print(json.dumps({"metric": "Eq. 27 vs Eq. 20 accuracy (periodic Taylor-Green 512^2)",
                              "rows": lumped_accuracy(cg, torch)}), flush=True)
        if args.jobelin:
            print(json.dumps({"metric": "Jobelin vortex errors and CGP speedup (paper Sections 3.2-3.3)",
                              "rows": jobelin_tables(cg, torch)}), flush=True)
        if args.c5:
            print(json.dumps(c5_study(cg, torch)), flush=True)
        return 0
    if args.batch_only:
        if rank != 0:
            return 0
        import torch
        from paper_1812_00185_gb300 import binding as cg
        print(json.dumps(batch_throughput(cg, torch, args.batch, args.batch_steps, args.warmup, args.batch_cluster,
                                          args.batch_threads, args.tol_inner)), flush=True)
        return 0
    if args.pcg_only:
        if rank != 0:
            return 0
        import torch
        from paper_1812_00185_gb300 import binding as cg
        peak, _ = _peaks()
        for n in args.pcg_n:
            print(json.dumps(pcg_bandwidth(cg, torch, n, peak)), flush=True)
            if n >= 2048:
                print(json.dumps(transfer_bandwidth(cg, torch, n, peak)), flush=True)
        return 0

    if world > 1:
        import torch
        import torch.distributed as dist
        torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", "0")))
        dist.init_process_group("nccl")
    out, (w, base) = run_gpu(args, rank, world)
    if world > 1:
        aggregate_ranks(out, world, "cuda")
    if rank == 0:
        print(json.dumps(out))
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
