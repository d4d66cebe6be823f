"""Autotuner for the Fock-build tile shapes and launch parameters, and the batched-SCF slot
count.

The library exposes its launch choices as named knobs (df_tune_set / df_tune_get): tile
shapes (the FP64 half-transform's column tile, the tcgen05 half-transform's tile width, the
auxiliary rows per CTA of J's first pass and per slice of its second), the tcgen05 GEMM's
shared-memory ring depth and the K-dimension splits of the exchange SYRK (tensor-core and
FP64).  This module times df_jk with CUDA events on the caller's stream for candidate
values (coordinate descent: one knob at a time, keeping the best), and stores the winners in
a JSON cache keyed by a problem-size bucket, so later runs of the same size class reuse
them.  Batched SCF has its own entry, tuned on molecules/s with many molecules in flight.
`python -m paper_2506_06661_gb300.tune` fills the buckets of the batched workload's size
range (nao 50-400) in both precisions and the batched-SCF entry.
"""
from __future__ import annotations

import ctypes
import json
import math
import os

import torch

from . import _check, lib

CACHE = os.environ.get("DFSCF_TUNE_CACHE", os.path.join(os.path.dirname(os.path.abspath(__file__)), "tune_cache.json"))

# The CTA-pair exchange SYRK (knob syrk_pair) is not searched: it is for single-stream Fock
# builds only (a batch with many molecules in flight stalled with it), and the cache enables it
# for the 300-centre bucket by hand.
# Launch parameters and tile shapes searched per precision: FP64 half-transform tile columns,
# tcgen05 half-transform tile width (0 = widest that fits) and ring depth, K-dimension splits
# of the exchange SYRK, auxiliary rows per slice / per CTA of J's passes.
CANDIDATES = {
    "fp64": {"fp64_ht_cols": [16, 32], "fp64_syrk_split": [0, 4, 9, 18, 36], "jpass2_rows": [128, 256, 512],
             "jpass1_rows": [1, 2]},
    "mixed": {"ht_n": [0, 64, 128], "syrk_bk": [32, 16], "umma_max_stages": [2, 4, 8],
              "syrk_split": [0, 16, 44, 88, 176],
              "jpass2_rows": [128, 256, 512], "jpass1_rows": [1, 2]},
}

# Representative molecules of the batched workload's size range (nao 50-400): one per
# power-of-two bucket of nao.
BUCKET_CENTRES = (10, 20, 40, 80)


# Knobs searched for batched-SCF throughput (many molecules in flight share the SMs, so the
# best single-molecule launch shapes are not the best here).
BATCH_CANDIDATES = {"syrk_split": [0, 44], "umma_max_stages": [8, 2], "ht_n": [0, 128], "jpass1_rows": [1, 2]}


def reset() -> None:
    """Every knob back to its built-in value."""
    lib().df_tune_reset()


def set_knob(name: str, value: int) -> None:
    _check(lib().df_tune_set(name.encode(), int(value)))


def get_knob(name: str) -> int:
    return int(lib().df_tune_get(name.encode()))


def bucket(nao: int, naux: int, nocc: int, precision: str) -> str:
    p2 = lambda x: 1 << max(0, math.ceil(math.log2(max(1, x))))  # noqa: E731
    return f"{precision}:nao{p2(nao)}:naux{p2(naux)}:nocc{p2(nocc)}"


def load_cache(path: str = CACHE) -> dict:
    try:
        with open(path) as fh:
            return json.load(fh)
    except (OSError, ValueError):
        return {}


def save_cache(cache: dict, path: str = CACHE) -> None:
    tmp = path + ".tmp"
    with open(tmp, "w") as fh:
        json.dump(cache, fh, indent=1, sort_keys=True)
    os.replace(tmp, path)


def apply(key: str, cache: dict | None = None) -> dict:
    """Set the knobs stored for `key`; returns them ({} when the bucket is not cached)."""
    c = load_cache() if cache is None else cache
    knobs = c.get(key, {}).get("knobs", {})
    for k, v in knobs.items():
        set_knob(k, v)
    return knobs


def _time_jk(dfscf, B, D, C, precision: str, reps: int) -> float:
    work = dfscf.JKWorkspace(B.nao, B.naux, C.shape[1], precision)
    J = torch.empty_like(D)
    K = torch.empty_like(D)
    dfscf.jk(B, D, C, precision=precision, work=work, out_j=J, out_k=K)
    s = torch.cuda.current_stream()
    times = []
    for _ in range(reps):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(s)
        dfscf.jk(B, D, C, precision=precision, work=work, out_j=J, out_k=K)
        e1.record(s)
        torch.cuda.synchronize()
        times.append(e0.elapsed_time(e1))
    del work
    return sorted(times)[len(times) // 2]


def tune_fock(B, D, C, precision: str = "mixed", reps: int = 3, log=None) -> dict:
    """Coordinate descent over the knobs of `precision`; returns {knobs, ms, baseline_ms}."""
    import paper_2506_06661_gb300 as dfscf
    cands = CANDIDATES[precision]
    best = {k: get_knob(k) for k in cands}
    for k, v in best.items():
        set_knob(k, v)
    base = _time_jk(dfscf, B, D, C, precision, reps)
    best_ms = base
    for name, values in cands.items():
        for v in values:
            if v == best[name]:
                continue
            set_knob(name, v)
            ms = _time_jk(dfscf, B, D, C, precision, reps)
            if log:
                log(f"  {name}={v}: {ms:.3f} ms")
            if ms < best_ms * 0.995:
                best_ms, best[name] = ms, v
            set_knob(name, best[name])
    return {"knobs": best, "ms": best_ms, "baseline_ms": base}


def tune_and_store(B, D, C, nocc: int, precision: str, reps: int = 3, log=None) -> dict:
    key = bucket(B.nao, B.naux, nocc, precision)
    res = tune_fock(B, D, C, precision, reps, log)
    cache = load_cache()
    cache[key] = res
    save_cache(cache)
    return {"key": key, **res}


def tune_batch_slots(mols, precision: str = "mixed", candidates=(16, 32, 64), sample: int = 64) -> dict:
    """Slots (molecules in flight) that give the highest molecules/s on a sample."""
    import time
    import paper_2506_06661_gb300 as dfscf
    devs = [dfscf.MoleculeOnDevice(m) for m in mols[:sample]]
    out = {}
    for s in candidates:
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        dfscf.scf_run_batch(devs, slots=s, precision=precision, raise_on_noconv=False)
        torch.cuda.synchronize()
        out[s] = len(devs) / (time.perf_counter() - t0)
    best = max(out, key=out.get)
    cache = load_cache()
    entry = cache.get(f"batch:{precision}", {})
    entry.update({"slots": best, "molecules_per_s": out})
    cache[f"batch:{precision}"] = entry
    save_cache(cache)
    return {"slots": best, "molecules_per_s": out}


def tune_batch_knobs(mols, precision: str = "mixed", slots: int = 128, sample: int = 64, log=None) -> dict:
    """Coordinate descent over BATCH_CANDIDATES on the molecules/s of scf_run_batch over a
    sample (from the built-in values; a change must gain 3%); stored as the "knobs" of the
    cache entry "batch:<precision>"."""
    import time
    import paper_2506_06661_gb300 as dfscf
    devs = [dfscf.MoleculeOnDevice(m) for m in mols[:sample]]
    reset()

    def rate():
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        dfscf.scf_run_batch(devs, slots=slots, precision=precision, raise_on_noconv=False)
        torch.cuda.synchronize()
        return len(devs) / (time.perf_counter() - t0)

    rate()  # first run: graph capture and lazy module loads
    best = {k: get_knob(k) for k in BATCH_CANDIDATES}
    base = best_rate = rate()
    for name, values in BATCH_CANDIDATES.items():
        for v in values:
            if v == best[name]:
                continue
            set_knob(name, v)
            r = rate()
            if log:
                log(f"  batch {name}={v}: {r:.3f} molecules/s")
            if r > best_rate * 1.03:
                best_rate, best[name] = r, v
            set_knob(name, best[name])
    cache = load_cache()
    entry = cache.get(f"batch:{precision}", {})
    entry.update({"knobs": best, "molecules_per_s_sample": best_rate, "baseline_per_s_sample": base,
                  "sample": len(devs), "slots_tuned_with": slots})
    cache[f"batch:{precision}"] = entry
    save_cache(cache)
    return entry


def apply_batch(precision: str = "mixed") -> dict:
    """Built-in knob values, then those stored for batched SCF ({} when none are cached)."""
    reset()
    return apply(f"batch:{precision}")


def tune_buckets(precision: str = "mixed", centres=BUCKET_CENTRES, reps: int = 3, log=None) -> dict:
    """Tune the knobs for one representative molecule per size bucket (seed 0, one centre per
    10 bohr^3, core-guess density) and store each bucket's winners in the cache."""
    import gen
    import paper_2506_06661_gb300 as dfscf
    out = {}
    for n in centres:
        mol = gen.make_molecule(n, gen.molecules.box_for(n), 0)
        md = dfscf.MoleculeOnDevice(mol)
        L = dfscf.metric_chol(mol.aux_xyz, mol.aux_exp)
        B = dfscf.build_B(mol.ao_xyz, mol.ao_exp, mol.aux_xyz, mol.aux_exp, L, precision)
        C, D, *_ = dfscf.core_guess(md)
        res = tune_and_store(B, D, C, mol.nocc, precision, reps, log)
        out[res["key"]] = res
        del B
    return out


def apply_for_molecules(mols, precision: str) -> dict:
    """Apply the cached knobs of the bucket of the largest molecule (it dominates the work of
    a batch); returns them ({} when that bucket is not cached)."""
    big = max(mols, key=lambda m: m.nao)
    return apply(bucket(big.nao, big.naux, big.nelec // 2, precision))


if __name__ == "__main__":
    import sys
    import gen
    for prec in ("mixed", "fp64"):
        for k, v in tune_buckets(prec, log=print).items():
            print(k, v["knobs"], f"{v['baseline_ms']:.3f} -> {v['ms']:.3f} ms", flush=True)
    e = tune_batch_knobs(gen.batch_molecules(256, 10, 80, 1), "mixed", log=print)
    print("batch:mixed", e["knobs"], f"{e['baseline_per_s_sample']:.3f} -> {e['molecules_per_s_sample']:.3f} "
          "molecules/s", flush=True)
    sys.exit(0)
