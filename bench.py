"""Benchmark: density-fitted Fock builds (J + K) on the 300-centre workload.

Workload (default): 300 hydrogen-like centres at one per 10 bohr^3 (box 14.42 bohr,
seed 0), 5 orbital + 15 auxiliary s primitives per centre: nao 1500, naux 4500,
nocc 150; D and C_occ from the core-Hamiltonian guess, fixed.  One step is one Fock
build (J[D] and K[C_occ]) in FP64; the mixed-precision build (K from split-BF16 planes on
tcgen05 tensor cores, J in FP64) is timed the same way and reported under "mixed".  B (40.5 GB FP64) is far larger
than L2, so no L2 flush is needed between steps.

--impl reference times the CPU oracle (the plain FP64 C loops in oracle/) on a bounded
P-slice of the same workload and scales it to one full build.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "DF-JK builds/s + tensor-pipe %; SCF time-to-1e-6 Eh, mixed vs FP64"
# FP64 ALU peak: 152 SMs x 2 FP64 FMA/clk/SM x 2 flop x 2.07 GHz (1.90 FMA/clk/SM measured)
FP64_PEAK_TFLOPS = 152 * 2 * 2 * 2.07e9 / 1e12
LAUNCHES_FP64 = 7   # kernels per FP64 build: Dw, J pass 1, J pass 2, J reduce, K half-transform, K SYRK, K mirror
LAUNCHES_MIXED = 9  # Dw, J pass 1, J pass 2, J reduce, C^T planes, tcgen05 half-transform, X planes, tcgen05 SYRK,
#                     K reduce


def load_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as fh:
            return json.load(fh), "measured"
    except OSError:
        return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "bf16_tflops_sustained": 1700.0}, "fallback"


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled every 200 ms during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.idx = gpu_index
        self.proc = None

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.idx), f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except OSError:
            self.proc = None
        return self

    def __exit__(self, *a):
        self.lines = []
        if self.proc is not None:
            self.proc.terminate()
            try:
                out, _ = self.proc.communicate(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()
                out, _ = self.proc.communicate()
            self.lines = [l for l in out.splitlines() if l.strip()]

    def summary(self):
        sm, mx, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for l in getattr(self, "lines", []):
            f = [x.strip() for x in l.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                mx = float(f[2])
            except ValueError:
                continue
            for nm, v in zip(names, f[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": mx, "reasons": sorted(reasons),
                "samples": len(sm)}


def workload(name: str):
    import gen
    if name == "c1":
        return gen.config_c1(), "300 H centres, 1 per 10 bohr^3 (box 14.42 bohr, seed 0); nao 1500, naux 4500, nocc 150"
    if name == "c0":
        return gen.config_c0(), "20 H centres in a 6 bohr cube (seed 0); nao 100, naux 300, nocc 10"
    if name in ("m80", "m120"):
        n = int(name[1:])
        return gen.make_molecule(n, gen.molecules.box_for(n), 0), \
            f"{n} H centres, 1 per 10 bohr^3 (seed 0); nao {5 * n}, naux {15 * n}, nocc {n // 2}"
    raise SystemExit(f"unknown workload {name}")


def max_over_ranks(x: float, device: str = "cuda") -> float:
    """Maximum of a per-rank value over all ranks (identity without torch.distributed)."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return x
    t = torch.tensor([x], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def dist_env():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


# ---------------------------------------------------------------------------------------
def cpu_oracle_sample(mol, rows: int):
    """Time the oracle's DF-J and DF-K on `rows` auxiliary rows; returns (seconds, rows).
    The raw three-centre rows stand in for B: the oracle's loop cost does not depend on
    the values."""
    import oracle
    oracle.build_library()
    R = oracle.int3c(mol.ao_xyz, mol.ao_exp, mol.aux_xyz[:rows], mol.aux_exp[:rows])
    rng = np.random.default_rng(0)
    C = 0.05 * rng.standard_normal((mol.nao, mol.nocc))
    D = 2 * C @ C.T
    t0 = time.perf_counter()
    oracle.df_j(R, mol.nao, D)
    oracle.df_k(R, mol.nao, C)
    return time.perf_counter() - t0


def cpu_cores():
    try:
        return len(os.sched_getaffinity(0))
    except AttributeError:
        return os.cpu_count() or 1


def cpu_model() -> str:
    """The host CPU's model name (lscpu, else /proc/cpuinfo)."""
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for line in out.splitlines():
            if line.strip().startswith("Model name:"):
                return line.split(":", 1)[1].strip()
    except (OSError, subprocess.SubprocessError):
        pass
    try:
        with open("/proc/cpuinfo") as fh:
            for line in fh:
                if line.lower().startswith("model name"):
                    return line.split(":", 1)[1].strip()
    except OSError:
        pass
    return "unknown"


def oracle_threads(n: int) -> None:
    """Thread count of the oracle library's OpenMP loops."""
    import ctypes
    import oracle
    f = oracle.lib().omp_set_num_threads
    f.argtypes = [ctypes.c_int]
    f(int(n))


def cpu_b_build_sample(mol):
    """Oracle B build on the host: the full metric and its Cholesky factor, then the
    3-centre rows of orbitals 0 and 1 (2 nao columns of the pair index) whitened by forward
    substitution; the column part scaled to npair columns.  Returns (seconds estimate, text)."""
    import oracle
    t0 = time.perf_counter()
    L = oracle.cholesky(oracle.int2c(mol.aux_xyz, mol.aux_exp))
    t1 = time.perf_counter()
    R = oracle.int3c_rows(mol.ao_xyz, mol.ao_exp, mol.aux_xyz, mol.aux_exp, [0, 1])
    oracle.whiten(L, R.reshape(R.shape[0], -1))
    t2 = time.perf_counter()
    ncol = R.shape[1] * R.shape[2]
    npair = mol.nao * (mol.nao + 1) // 2
    est = (t1 - t0) + (t2 - t1) * npair / ncol
    return est, (f"metric + Cholesky {t1 - t0:.1f} s, then {ncol} of {npair} pair columns integrated and whitened "
                 f"in {t2 - t1:.1f} s, scaled to all columns")


def cpu_baseline_obj(mol, wl_name):
    cores = cpu_cores()
    rows = min(mol.naux, 12 * cores)
    t = cpu_oracle_sample(mol, rows)
    per_build = t * mol.naux / rows
    out = {"value": 1.0 / per_build, "unit": "builds/s", "cores": cores, "kind": "oracle",
           "sample": f"oracle DF-J + DF-K over the first {rows} of {mol.naux} auxiliary rows of the {wl_name} "
                     f"workload ({t:.1f} s), scaled linearly in naux to one full Fock build",
           "cpu_model": cpu_model()}
    # one core: the same loops with one OpenMP thread on a smaller slice
    rows1 = min(mol.naux, 6)
    oracle_threads(1)
    try:
        t1 = cpu_oracle_sample(mol, rows1)
    finally:
        oracle_threads(cores)
    out["one_core"] = {"value": rows1 / (t1 * mol.naux), "unit": "builds/s",
                       "sample": f"{rows1} auxiliary rows on one thread ({t1:.1f} s), scaled to one full build"}
    est, text = cpu_b_build_sample(mol)
    out["b_build"] = {"seconds_estimate": est, "cores": cores, "sample": text}
    return out


def run_reference(args):
    ws, rank, _ = dist_env()
    if rank != 0:
        return 0
    mol, desc = workload(args.workload)
    cores = cpu_cores()
    rows = min(mol.naux, max(1, 4 * cores))
    for _ in range(args.warmup):
        cpu_oracle_sample(mol, rows)
    times = [cpu_oracle_sample(mol, rows) * mol.naux / rows for _ in range(args.steps)]
    ms = 1000.0 * statistics.mean(times)
    v = 1000.0 / ms
    line = {"impl": "reference", "metric": METRIC, "value": v, "unit": "builds/s", "n_gpus": ws, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": desc, "precision": "fp64"},
            "cpu_baseline": {"value": v, "unit": "builds/s", "cores": cores, "kind": "oracle",
                             "sample": f"each step: oracle DF-J + DF-K over {rows} of {mol.naux} auxiliary rows, "
                                       f"scaled linearly in naux to one full Fock build"},
            "e2e": {"value": v, "unit": "builds/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


# ---------------------------------------------------------------------------------------
def time_builds(dfscf, torch, B, D, C, prec, steps, warmup, work, barrier):
    stream = torch.cuda.current_stream()
    J = torch.empty_like(D)
    K = torch.empty_like(D)
    for _ in range(warmup):
        dfscf.jk(B, D, C, precision=prec, work=work, out_j=J, out_k=K)
    barrier()
    torch.cuda.synchronize()
    dfscf.profile_reset()
    dfscf.profile_enable(True)
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    torch.cuda.nvtx.range_push(f"fock_{prec}")  # lets a profiler select the timed builds
    e0.record(stream)
    for _ in range(steps):
        dfscf.jk(B, D, C, precision=prec, work=work, out_j=J, out_k=K)
    e1.record(stream)
    torch.cuda.nvtx.range_pop()
    torch.cuda.synchronize()
    dfscf.profile_enable(False)
    prof = dfscf.profile_read()
    barrier()
    return e0.elapsed_time(e1) / steps, prof


def time_e2e(dfscf, torch, B, D, C, prec, steps, work):
    """Host-buffer Fock builds: pinned D, C copied in, J, K copied out, inside the timed region."""
    nao, nocc = D.shape[0], C.shape[1]
    hD = torch.empty(nao, nao, dtype=torch.float64, pin_memory=True).copy_(D.cpu())
    hC = torch.empty(nao, nocc, dtype=torch.float64, pin_memory=True).copy_(C.cpu())
    hJ = torch.empty(nao, nao, dtype=torch.float64, pin_memory=True)
    hK = torch.empty(nao, nao, dtype=torch.float64, pin_memory=True)
    dD, dC = torch.empty_like(D), torch.empty_like(C)
    J, K = torch.empty_like(D), torch.empty_like(D)
    stream = torch.cuda.current_stream()

    def one():
        dD.copy_(hD, non_blocking=True)
        dC.copy_(hC, non_blocking=True)
        dfscf.jk(B, dD, dC, precision=prec, work=work, out_j=J, out_k=K)
        hJ.copy_(J, non_blocking=True)
        hK.copy_(K, non_blocking=True)

    one()
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(steps):
        one()
    e1.record(stream)
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / steps
    return ms, (hD.numel() + hC.numel()) * 8, (hJ.numel() + hK.numel()) * 8


def roofline_of(prof, name, flops_per_launch=None, bytes_per_launch=None, peak=None, bound="alu", unit="TFLOP/s"):
    if name not in prof:
        return None
    ms, calls = prof[name]
    avg = ms / max(calls, 1)
    if flops_per_launch is not None:
        ach = flops_per_launch / (avg * 1e-3) / 1e12
    else:
        ach = bytes_per_launch / (avg * 1e-3) / 1e9
    return {"kernel": name, "bound": bound, "achieved": ach, "peak": peak, "unit": unit, "frac": ach / peak,
            "traffic": None, "avg_ms": avg, "launches": calls}


def scf_time_to_convergence(dfscf, torch, wl, oracle_energy=False, max_cycle=100):
    """Wall time, iterations and energies of the mixed-precision and the plain FP64 SCF of
    one molecule (one untimed warm-up run each builds and captures the graphs first)."""
    mol, desc = workload(wl)
    md = dfscf.MoleculeOnDevice(mol)
    out = {"workload": desc}
    for prec in ("mixed", "fp64"):
        work = dfscf._work(dfscf.scf_work_bytes(md.nao, md.naux, md.nelec // 2, prec))
        dfscf.scf_run(md, precision=prec, work=work, raise_on_noconv=False, max_cycle=max_cycle)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        r = dfscf.scf_run(md, precision=prec, work=work, raise_on_noconv=False, max_cycle=max_cycle)
        torch.cuda.synchronize()
        out[prec] = {"seconds": time.perf_counter() - t0, "energy": r.energy, "iterations": r.iterations,
                     "fp64_iterations": r.fp64_iterations, "converged": r.converged}
        del work
    out["abs_dE_mixed_vs_fp64"] = abs(out["mixed"]["energy"] - out["fp64"]["energy"])
    out["speedup_mixed_over_fp64"] = out["fp64"]["seconds"] / out["mixed"]["seconds"]
    if oracle_energy:
        from oracle import scf as oscf
        e = oscf.rhf(oscf.build_system(mol)).energy
        out["oracle_energy"] = e
        for prec in ("mixed", "fp64"):
            out[prec]["abs_err_vs_oracle"] = abs(out[prec]["energy"] - e)
    return out


def run_ours(args):
    import torch
    ws, rank, local = dist_env()
    if ws > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl" if torch.cuda.is_available() else "gloo")
        barrier = dist.barrier
    else:
        def barrier():
            return None
    torch.cuda.set_device(local)
    import paper_2506_06661_gb300 as dfscf
    peaks, peak_src = load_peaks()
    mol, desc = workload(args.workload)
    t_setup = time.perf_counter()
    md = dfscf.MoleculeOnDevice(mol)
    L = dfscf.metric_chol(mol.aux_xyz, mol.aux_exp)
    B = dfscf.build_B(mol.ao_xyz, mol.ao_exp, mol.aux_xyz, mol.aux_exp, L, "mixed" if args.mixed else "fp64")
    C, D, *_ = dfscf.core_guess(md)
    if args.kcols > 0:
        # exchange over kcols seeded columns instead of C_occ: profiles the tile width of a
        # larger molecule's occupied space on a smaller B
        g = torch.Generator(device="cpu").manual_seed(args.kcols)
        C = (torch.randn(mol.nao, args.kcols, generator=g, dtype=torch.float64) / mol.nao ** 0.5).to("cuda")
    torch.cuda.synchronize()
    t_setup = time.perf_counter() - t_setup
    nao, naux, nocc = mol.nao, mol.naux, C.shape[1]
    npair = nao * (nao + 1) // 2
    # launch knobs: the autotuner's cached winners for this size bucket (or a fresh tuning
    # with --tune, stored in the cache), else the library defaults
    from paper_2506_06661_gb300 import tune
    knobs = {}
    for prec in ("fp64", "mixed") if args.mixed else ("fp64",):
        key = tune.bucket(nao, naux, nocc, prec)
        if args.tune:
            res = tune.tune_and_store(B, D, C, nocc, prec)
            knobs[prec] = {"bucket": key, "source": "tuned now", **res["knobs"]}
        else:
            got = tune.apply(key)
            knobs[prec] = {"bucket": key, "source": "tune cache" if got else "defaults", **got}
    for kv in args.knob:
        name, val = kv.split("=")
        tune.set_knob(name, int(val))
        knobs.setdefault("forced", {})[name] = int(val)
    work64 = dfscf.JKWorkspace(nao, naux, nocc, "fp64")

    with ClockSampler(local) as clk:
        ms64, prof64 = time_builds(dfscf, torch, B, D, C, "fp64", args.steps, args.warmup, work64, barrier)
    clocks = clk.summary()

    # max over ranks of the per-step time; every rank ran the same number of builds
    ms64 = max_over_ranks(ms64)
    value = ws * 1000.0 / ms64

    ht_flops = 2.0 * naux * nao * nao * nocc
    syrk_flops = 1.0 * naux * nocc * nao * nao
    j_bytes = 8.0 * naux * dfscf.lib().df_B_ld(nao)
    rl = {}
    for name, fl in (("k_halftransform_fp64", ht_flops), ("k_syrk_fp64", syrk_flops)):
        r = roofline_of(prof64, name, flops_per_launch=fl, peak=FP64_PEAK_TFLOPS, bound="alu")
        if r:
            rl[name] = r
    for name in ("j_pass1", "j_pass2"):
        r = roofline_of(prof64, name, bytes_per_launch=j_bytes, peak=peaks["hbm_gbs"], bound="hbm", unit="GB/s")
        if r:
            rl[name] = r
    dominant = max(rl.values(), key=lambda r: r["avg_ms"] * r["launches"]) if rl else None
    # DRAM traffic of the FP64 half-transform: the ncu capture of the same kernel (32
    # occupied columns per CTA, the variant this workload runs) on the 80-centre workload
    # read 772.81 MB and wrote 144.74 MB against 926.0 MB of algorithmic bytes (B read once,
    # X written once); traffic grows with those bytes, so one launch here moves that ratio
    # times its own algorithmic bytes
    if dominant and dominant["kernel"] == "k_halftransform_fp64":
        ht_bytes = 8.0 * naux * dfscf.lib().df_B_ld(nao) + 8.0 * nao * naux * nocc
        m80_bytes = 8.0 * 1200 * dfscf.lib().df_B_ld(400) + 8.0 * 400 * 1200 * 40
        dominant["traffic"] = (772.808448e6 + 144.741120e6) / m80_bytes * ht_bytes
        dominant["traffic_source"] = ("ncu dram__bytes_read.sum + dram__bytes_write.sum of the 80-centre capture, "
                                      "scaled by the algorithmic bytes of this launch")

    e2e_ms, h2d, d2h = time_e2e(dfscf, torch, B, D, C, "fp64", args.e2e_steps, work64)

    mixed = None
    if args.mixed:
        workm = dfscf.JKWorkspace(nao, naux, nocc, "mixed")
        with ClockSampler(local) as clkm:
            msm, profm = time_builds(dfscf, torch, B, D, C, "mixed", args.mixed_steps, args.warmup, workm, barrier)
        # accuracy of this build against the FP64 build of the same inputs
        Jm, Km = dfscf.jk(B, D, C, precision="mixed", work=workm)
        J6, K6 = dfscf.jk(B, D, C, precision="fp64", work=work64)
        errj = float((Jm - J6).abs().max() / J6.abs().max())
        errk = float((Km - K6).abs().max() / K6.abs().max())
        npad = dfscf.lib().df_nao_pad(nao)
        ncpad = max(16, (nocc + 15) // 16 * 16)
        planes = int(dfscf.lib().df_tune_get(b"mixed_planes"))
        products = planes * (planes + 1) // 2
        bk = 32 if planes >= 4 else 64                       # K box of the tcgen05 ring
        max_n = min(256, ((220 * 1024 // 2) // planes - 128 * bk * 2) // (bk * 2) // 16 * 16)
        ntc = -(-ncpad // max_n)
        nht = (-(-ncpad // ntc) + 15) // 16 * 16
        # tensor-core flops issued (padded tiles) and the algorithmic count of the same products
        tc_ht = products * 2.0 * naux * npad * npad * (nht * ntc)
        syrk_n = 128                                          # 128 x 128 tiles (4 accumulators)
        nblk = npad // 128
        if int(dfscf.lib().df_tune_get(b"syrk_pair")):
            # CTA pairs: 256 x 128 blocks up to each double row's diagonal, two tiles each
            syrk_tiles = 2 * sum(min(2 * mp + 2, nblk) for mp in range((nblk + 1) // 2))
        else:
            syrk_tiles = nblk * (nblk + 1) // 2                # lower 128 x 128 tiles
        tc_syrk = products * 2.0 * (naux * ncpad) * (128 * syrk_n) * syrk_tiles
        rlm = {}
        for name, fl, alg in (("k_halftransform_tc", tc_ht, products * ht_flops),
                              ("k_syrk_tc", tc_syrk, products * syrk_flops)):
            r = roofline_of(profm, name, flops_per_launch=alg, peak=peaks["bf16_tflops_sustained"], bound="tensor")
            if r:
                r["issued_tflops"] = fl / (r["avg_ms"] * 1e-3) / 1e12
                r["issued_frac"] = r["issued_tflops"] / peaks["bf16_tflops_sustained"]
                rlm[name] = r
        for name in ("j_pass1", "j_pass2"):
            r = roofline_of(profm, name, bytes_per_launch=j_bytes, peak=peaks["hbm_gbs"], bound="hbm", unit="GB/s")
            if r:
                rlm[name] = r
        mixed = {"value": ws * 1000.0 / msm, "unit": "builds/s", "ms_per_step": msm, "steps": args.mixed_steps,
                 "dtype": f"bf16 planes x{planes}, {products} products, two fixed-point planes, exact fp32 sums of their products (K); f64 (J)",
                 "rel_err_vs_fp64": {"J": errj, "K": errk},
                 "kernels": rlm, "gpu_launches": LAUNCHES_MIXED * args.mixed_steps, "clocks": clkm.summary(),
                 "phase_ms": {k: v[0] / max(v[1], 1) for k, v in profm.items()}}

    scf = None
    tune.reset()  # the SCF and batch blocks do not inherit this workload's launch knobs
    # nor its device memory: B alone holds 40.5 GB (FP64) plus the BF16 planes
    B = work64 = workm = Jm = Km = J6 = K6 = None
    torch.cuda.synchronize()
    torch.cuda.empty_cache()
    if not args.no_scf:
        scf = {"what": "wall time of scf_run to |dE| < 1e-8 Eh and max|e| < 1e-5 (integrals, metric, B and the "
                       "iterations), mixed precision against plain FP64, same molecule and options"}
        for wl in ("c0", "m120"):
            scf[wl] = scf_time_to_convergence(dfscf, torch, wl, oracle_energy=(wl == "c0"))
    batch = None
    if not args.no_batch:
        import gen
        mols = gen.batch_molecules(args.nmol, 10, 80, 1)
        devs = [dfscf.MoleculeOnDevice(m) for m in mols]
        from paper_2506_06661_gb300 import tune
        batch_knobs = tune.apply_batch("mixed")
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        res = dfscf.scf_run_batch(devs, slots=args.batch_slots, precision="mixed", raise_on_noconv=False).results
        torch.cuda.synchronize()
        dt = time.perf_counter() - t0
        batch = {"workload": f"{len(mols)} molecules of 10-80 H centres (uniform size draw, seed 1; nao 50-400), "
                             "mixed-precision SCF to |dE| < 1e-8 Eh and max|e| < 1e-5",
                 "seconds": dt, "molecules_per_s": len(mols) / dt, "converged": int(sum(r.converged for r in res)),
                 "mean_iterations": float(np.mean([r.iterations for r in res])),
                 "mean_fp64_iterations": float(np.mean([r.fp64_iterations for r in res])),
                 "max_in_flight": args.batch_slots, "knobs": batch_knobs or "library defaults"}
        # the same batch with the stability analysis of every solution and the escape from
        # saddle points (knob stability = 2), so that every molecule ends in a minimum
        tune.set_knob("stability", 2)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        res2 = dfscf.scf_run_batch(devs, slots=args.batch_slots, precision="mixed", raise_on_noconv=False).results
        torch.cuda.synchronize()
        dt2 = time.perf_counter() - t0
        tune.set_knob("stability", 0)
        hm = np.array([r.hess_min for r in res2], dtype=float)
        batch["with_saddle_escape"] = {
            "seconds": dt2, "molecules_per_s": len(mols) / dt2, "converged": int(sum(r.converged for r in res2)),
            "saddle_escapes": int(sum(r.stability_restarts for r in res2)),
            "min_hess_min": float(np.nanmin(hm)) if np.isfinite(hm).any() else None,
            "negative_hess_min": int(np.sum(hm < 0))}
        del devs

    line = {"metric": METRIC, "value": value, "unit": "builds/s", "n_gpus": ws, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms64, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": desc, "precision": "fp64", "step": "one Fock build: J[D] and K[C_occ]",
                       "knobs": knobs,
                       "l2": "inputs larger than L2 (B is %.1f GB)" % (8.0 * naux * npair / 1e9),
                       "parallelism": f"replicas x{ws}" if ws > 1 else "single GPU"},
            "roofline": ({k: v for k, v in dominant.items() if k not in ("avg_ms", "launches")} | {"peak_source": (
                "derived FP64 ALU peak: 152 SMs x 2 FMA/clk x 2 flop x 2.07 GHz" if dominant["bound"] == "alu"
                else f"MEASURED_PEAKS.json ({peak_src})")}) if dominant else None,
            "kernels": rl,
            "phase_ms": {k: v[0] / max(v[1], 1) for k, v in prof64.items()},
            "e2e": {"value": ws * 1000.0 / e2e_ms, "unit": "builds/s", "h2d_bytes_per_step": h2d,
                    "d2h_bytes_per_step": d2h, "steps": args.e2e_steps},
            "gpu_launches": LAUNCHES_FP64 * args.steps,
            "clocks": clocks,
            "setup_s": t_setup,
            "mixed": mixed,
            "scf": scf,
            "batch": batch}
    if rank == 0 and ws == 1 and not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline_obj(mol, args.workload)
    if rank == 0:
        print(json.dumps(line), flush=True)
    if ws > 1:
        import torch.distributed as dist
        dist.destroy_process_group()
    return 0


def run_scenario_scf(args):
    """Time to convergence of the plain FP64 SCF and the mixed-precision SCF (same molecule)."""
    import torch
    import paper_2506_06661_gb300 as dfscf
    mol, desc = workload(args.workload)
    md = dfscf.MoleculeOnDevice(mol)
    out = {"scenario": "scf", "workload": desc}
    ref = None
    if args.workload == "c0":
        from oracle import scf as oscf
        ref = oscf.rhf(oscf.build_system(mol)).energy
        out["oracle_energy"] = ref
    for prec in ("mixed", "fp64"):
        work = dfscf._work(dfscf.scf_work_bytes(md.nao, md.naux, md.nelec // 2, prec))
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        r = dfscf.scf_run(md, precision=prec, work=work, raise_on_noconv=False, max_cycle=args.max_cycle)
        torch.cuda.synchronize()
        dt = time.perf_counter() - t0
        out[prec] = {"seconds": dt, "energy": r.energy, "iterations": r.iterations,
                     "fp64_iterations": r.fp64_iterations, "converged": r.converged, "last_dE": r.last_de,
                     "last_err": r.last_err}
        if args.phases:
            # a second, profiled run (graphs bypassed) gives the per-phase split of the time
            dfscf.profile_reset()
            dfscf.profile_enable(True)
            dfscf.scf_run(md, precision=prec, work=work, raise_on_noconv=False, max_cycle=args.max_cycle)
            dfscf.profile_enable(False)
            out[prec]["phase_ms_total"] = {k: round(v[0], 3) for k, v in dfscf.profile_read().items()}
        if ref is not None:
            out[prec]["abs_err_vs_oracle"] = abs(r.energy - ref)
        del work
    out["mixed_vs_fp64_abs_dE"] = abs(out["mixed"]["energy"] - out["fp64"]["energy"])
    out["speedup_mixed_over_fp64"] = out["fp64"]["seconds"] / out["mixed"]["seconds"]
    print(json.dumps(out), flush=True)
    return 0


def run_scenario_batch(args):
    """Batched SCF over molecules of 10-80 centres (uniform size draw, seed 1)."""
    import torch
    import gen
    import paper_2506_06661_gb300 as dfscf
    from paper_2506_06661_gb300 import tune
    mols = gen.batch_molecules(args.nmol, 10, 80, 1)
    devs = [dfscf.MoleculeOnDevice(m) for m in mols]
    slots, src = args.slots, "command line"
    if slots <= 0:
        # molecules in flight: the autotuner's choice (cached, else measured on a sample now)
        cached = tune.load_cache().get("batch:mixed")
        if cached and not args.tune:
            slots, src = int(cached["slots"]), "tune cache"
        else:
            t = tune.tune_batch_slots(mols, precision="mixed", candidates=(16, 32, 64), sample=64)
            slots, src = int(t["slots"]), f"tuned now on 64 molecules: {t['molecules_per_s']}"
    if args.tune:
        tune.tune_batch_knobs(mols, "mixed", slots=slots, log=print)
    knobs = tune.apply_batch("mixed")
    out = {"scenario": "batch", "molecules": len(mols), "centres": "10-80 (uniform, seed 1)",
           "nao_range": [min(m.nao for m in mols), max(m.nao for m in mols)], "slots": slots, "slots_source": src,
           "knobs": knobs or "library defaults"}
    per_mol = {}
    if args.stability:
        # lowest orbital-Hessian eigenvalue of every converged solution (Davidson), in the dump
        dfscf.lib().df_tune_set(b"stability", args.stability)
        out["stability"] = (f"{args.stability}: the times include the Davidson Hessian products"
                            + (" and the iterations after each saddle escape" if args.stability == 2 else ""))
    for prec in ("mixed",) + (("fp64",) if args.batch_fp64 else ()):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        res = dfscf.scf_run_batch(devs, slots=slots, precision=prec, raise_on_noconv=False).results
        torch.cuda.synchronize()
        dt = time.perf_counter() - t0
        conv = [r for r in res if r.converged]
        per_mol[prec] = res
        out[prec] = {"seconds": dt, "molecules_per_s": len(mols) / dt, "converged": len(conv),
                     "not_converged": [i for i, r in enumerate(res) if not r.converged],
                     "mean_iterations": float(np.mean([r.iterations for r in res])),
                     "mean_fp64_iterations": float(np.mean([r.fp64_iterations for r in res]))}
    if "fp64" in out:
        # the precision gap is judged on molecules that converged in both arms; the others
        # are listed by index
        both = [i for i in range(len(mols)) if per_mol["mixed"][i].converged and per_mol["fp64"][i].converged]
        d = np.array([abs(per_mol["mixed"][i].energy - per_mol["fp64"][i].energy) for i in both])
        out["converged_both"] = len(both)
        out["abs_dE_mixed_vs_fp64"] = {
            "max": float(d.max()) if d.size else None, "median": float(np.median(d)) if d.size else None,
            "over_1e-6": [both[k] for k in np.nonzero(d > 1e-6)[0]]}
    if args.dump:
        rows = []
        for i, m in enumerate(mols):
            row = {"index": i, "natm": m.natm, "nao": m.nao, "nelec": m.nelec}
            for prec, res in per_mol.items():
                r = res[i]
                row[prec] = {"energy": r.energy, "iterations": r.iterations, "fp64_iterations": r.fp64_iterations,
                             "converged": r.converged, "last_dE": r.last_de, "last_err": r.last_err,
                             "homo": r.homo, "lumo": r.lumo, "hess_min": r.hess_min,
                             "stability_restarts": r.stability_restarts}
            rows.append(row)
        with open(args.dump, "w") as fh:
            json.dump(rows, fh)
    print(json.dumps(out), flush=True)
    return 0


def run_scenario_guess(args):
    """Learned initial guess: train on converged SCFs of 10-40 centres (seed 2), evaluate
    mean iterations and wall time against the core guess on unseen 40-120-centre molecules (seed 3)."""
    import torch
    import gen
    from paper_2506_06661_gb300 import guess
    from paper_2506_06661_gb300 import tune
    slots = args.slots if args.slots > 0 else 32
    if args.load_model:
        # a model trained by an earlier run of this scenario (same recipe): evaluation only
        model = guess.GuessModel.load(args.load_model)
        train, ok, t_data, t_train, hist, nsamp = [], [], 0.0, 0.0, [None, None], 0
    else:
        t0 = time.perf_counter()
        train = gen.batch_molecules(args.ntrain, 10, 40, 2)
        # mixed precision ends with FP64 iterations, so the densities are FP64-converged
        res, Ds = guess.converged_densities(train, slots=slots, precision="mixed")
        ok = [i for i, r in enumerate(res) if r.converged]
        t_data = time.perf_counter() - t0
        X, Y, M = guess.build_dataset([train[i] for i in ok], [Ds[i] for i in ok])
        nsamp = int(M.sum().item())
        del Ds
        model = guess.GuessModel.create(seed=2)
        t0 = time.perf_counter()
        hist = guess.train(model, X, Y, M, epochs=args.epochs, batch=4096, lr=1e-3, seed=2)
        torch.cuda.synchronize()
        t_train = time.perf_counter() - t0
        if args.save_model:
            model.save(args.save_model)
    test = gen.batch_molecules(args.neval, 40, 120, 3)
    ev = guess.evaluate(model, test, slots=slots, precision="mixed")
    core_run = ev.pop("_core_run")
    for key in ("energy_core", "energy_learned", "iterations_core", "iterations_learned"):
        ev.pop(key, None)
    # the learned start's first exchange with coarser cuts of dm0's natural occupations
    cuts = {}
    for cut in [int(c) for c in args.dm0_cuts.split(",") if c]:
        old = tune.get_knob("dm0_eig_cut")
        tune.set_knob("dm0_eig_cut", cut)
        e2 = guess.evaluate(model, test, slots=slots, precision="mixed", core_run=core_run)
        tune.set_knob("dm0_eig_cut", old)
        cuts[f"1e-{cut}"] = {k: e2[k] for k in ("mean_iter_core", "mean_iter_learned", "same_state", "both_converged",
                                                "wall_s_core", "wall_s_learned", "guess_used")}
    ev["dm0_cuts"] = cuts
    # wider gates on the idempotency error of the predicted dm0 (default 1.0)
    gates = {}
    for gmax in [float(g) for g in args.guess_idem.split(",") if g]:
        old = tune.get_knob("guess_idem_max")
        tune.set_knob("guess_idem_max", int(round(100 * gmax)))
        e2 = guess.evaluate(model, test, slots=slots, precision="mixed", core_run=core_run)
        tune.set_knob("guess_idem_max", old)
        gates[f"{gmax:g}"] = {k: e2[k] for k in ("mean_iter_core", "mean_iter_learned", "same_state", "both_converged",
                                                 "wall_s_core", "wall_s_learned", "wall_s_predict", "guess_used",
                                                 "guess_rejected")}
    ev["idem_gates"] = gates
    out = {"scenario": "guess", "train_molecules": len(train), "train_converged": len(ok),
           "model": args.load_model or "trained in this run",
           "train_samples": nsamp, "data_seconds": t_data, "train_seconds": t_train,
           "epochs": args.epochs, "mse_first_last": [hist[0], hist[-1]], "eval_molecules": len(test),
           "eval_centres": "40-120 (uniform, seed 3)", "eval": ev}
    print(json.dumps(out), flush=True)
    return 0


def run_scenario_states(args):
    """SCF solutions reached by the FP64 and the mixed-precision runs of selected molecules of
    the batched workload, each tested by perturbation: the converged occupied orbitals are
    rotated by a small random angle into the virtual space (in the orthonormal basis of the
    overlap) and the FP64 SCF restarts from that determinant.  A local minimum comes back to
    its energy; a saddle point falls to a lower one.  The lowest orbital-Hessian eigenvalue of
    each solution (Davidson, knob "stability") is reported beside it: a small positive value is
    a soft mode, along which a loosely converged gradient leaves an energy error of about
    |g|^2 / (2 hess_min)."""
    import torch
    import gen
    import paper_2506_06661_gb300 as dfscf
    idx = [int(i) for i in args.indices.split(",") if i]
    sizes = gen.molecules.batch_sizes(256, 10, 80, 1)
    rng = np.random.default_rng(7)
    out = []
    dfscf.lib().df_tune_set(b"stability", 1)
    for i in idx:
        n = int(sizes[i])
        mol = gen.make_molecule(n, gen.molecules.box_for(n), (1, i))
        md = dfscf.MoleculeOnDevice(mol)
        S, _, _ = dfscf.int1e(mol.ao_xyz, mol.ao_exp, mol.xyz, mol.charges)
        S = S.cpu().numpy()
        s, U = np.linalg.eigh(S)
        X = U[:, s > 1e-8] / np.sqrt(s[s > 1e-8])
        row = {"index": i, "centres": n}
        for prec in ("fp64", "mixed"):
            r = dfscf.scf_run(md, precision=prec, raise_on_noconv=False)
            C = r.C.cpu().numpy()
            # orthonormal-basis occupied orbitals and their complement
            Cp = np.linalg.lstsq(X, C, rcond=None)[0]
            Q, _ = np.linalg.qr(np.hstack([Cp, rng.standard_normal((Cp.shape[0], Cp.shape[0] - Cp.shape[1]))]))
            Vp = Q[:, Cp.shape[1]:]
            probes = []
            for _ in range(args.probes):
                kappa = args.angle * rng.standard_normal((Vp.shape[1], Cp.shape[1])) / np.sqrt(Cp.shape[1])
                Cn, _ = np.linalg.qr(Cp + Vp @ kappa)
                Cao = X @ Cn[:, :Cp.shape[1]]
                rp = dfscf.scf_run(md, precision="fp64", dm0=2 * Cao @ Cao.T, raise_on_noconv=False)
                probes.append({"energy": rp.energy, "converged": rp.converged, "iterations": rp.iterations})
            lower = [p["energy"] for p in probes if p["converged"] and p["energy"] < r.energy - 1e-6]
            row[prec] = {"energy": r.energy, "converged": r.converged, "iterations": r.iterations,
                         "hess_min": r.hess_min, "last_err": r.last_err, "probes": probes, "minimum": not lower, "lowest_probe": min([p["energy"] for p in probes])}
        row["dE_mixed_minus_fp64"] = row["mixed"]["energy"] - row["fp64"]["energy"]
        out.append(row)
        print(json.dumps(row), flush=True)
    dfscf.lib().df_tune_set(b"stability", 0)
    return 0


def main():
    ap = argparse.ArgumentParser(description=__doc__)
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--workload", choices=["c1", "c0", "m80", "m120"], default="c1")
    ap.add_argument("--mixed-steps", type=int, default=20)
    ap.add_argument("--e2e-steps", type=int, default=3)
    ap.add_argument("--no-mixed", dest="mixed", action="store_false")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-scf", action="store_true", help="skip the SCF time-to-convergence block of the default line")
    ap.add_argument("--no-batch", action="store_true", help="skip the batched-SCF block of the default line")
    ap.add_argument("--kcols", type=int, default=0,
                    help="exchange over this many seeded columns instead of the occupied orbitals (profiling)")
    ap.add_argument("--batch-slots", type=int, default=128, help="molecules in flight in the batched-SCF block")
    ap.add_argument("--scenario", choices=["fock", "scf", "batch", "guess", "states"], default="fock",
                    help="fock: Fock-build throughput (the default line); scf: SCF time to convergence, "
                         "mixed vs FP64; batch: batched SCF of uneven molecules; guess: learned guess")
    ap.add_argument("--max-cycle", type=int, default=200, help="SCF iteration budget (scf, batch scenarios)")
    ap.add_argument("--phases", action="store_true", help="scf scenario: add a profiled run per precision")
    ap.add_argument("--nmol", type=int, default=256)
    ap.add_argument("--slots", type=int, default=0, help="molecules in flight (0: the autotuner's choice)")
    ap.add_argument("--tune", action="store_true", help="run the autotuner and store its winners in the cache")
    ap.add_argument("--knob", action="append", default=[], metavar="NAME=VALUE",
                    help="set a launch knob after the cached ones (repeatable)")
    ap.add_argument("--stability", type=int, default=0, choices=[0, 1, 2],
                    help="batch scenario: stability analysis of every converged solution (2: also leave saddles)")
    ap.add_argument("--batch-fp64", action="store_true")
    ap.add_argument("--ntrain", type=int, default=20000)
    ap.add_argument("--neval", type=int, default=512)
    ap.add_argument("--epochs", type=int, default=20)
    ap.add_argument("--save-model", default="")
    ap.add_argument("--load-model", default="", help="guess scenario: evaluate this saved model instead of training")
    ap.add_argument("--guess-idem", default="",
                    help="guess scenario: also evaluate these gates on the idempotency error of dm0 (e.g. 2,5)")
    ap.add_argument("--indices", default="2,6,156,214,246", help="states scenario: batch molecules to probe")
    ap.add_argument("--probes", type=int, default=4, help="states scenario: perturbed restarts per state")
    ap.add_argument("--angle", type=float, default=0.05, help="states scenario: rotation size (rad)")
    ap.add_argument("--dm0-cuts", default="", help="guess scenario: also evaluate these dm0_eig_cut exponents (e.g. 3,2)")
    ap.add_argument("--dump", default="", help="batch scenario: write per-molecule results to this JSON file")
    args = ap.parse_args()
    if args.scenario == "scf":
        return run_scenario_scf(args)
    if args.scenario == "batch":
        return run_scenario_batch(args)
    if args.scenario == "guess":
        return run_scenario_guess(args)
    if args.scenario == "states":
        return run_scenario_states(args)
    if args.impl == "reference":
        return run_reference(args)
    return run_ours(args)


if __name__ == "__main__":
    sys.exit(main())
