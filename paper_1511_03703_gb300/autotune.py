"""Autotuner for the ensemble CG launch knobs.

Knobs, all exposed through the C ABI:
  - SpMV arithmetic form per (mesh, s): native FP64 FMA, double-float on the
    FP32 pipe, alternate entries on each (ENS_CG_DF64 / ENS_CG_SPLIT64), or
    double-float on values pre-split once per ensemble (ens_cg_df);
    GB300's 1/64-rate FP64 makes the best form depend on s and mesh size;
  - SpMV mapping per (mesh, s, form): chunks of 32 rows per CTA
    (ENS_CG_K1_CHUNKS: 1, 2, 4 or 8, at most 1024 threads per CTA, each row on
    max(s/2, 2) threads), or one chunk per CTA with the upper levels of p.q's
    tree in a second kernel ("defer", ENS_CG_K1_DEFER), tuned jointly with the
    form; for a batch, the CTA size of the batched SpMV (ens_cg_batched,
    ENS_CG_BATCH_K1_WIDE);
  - graph length (check_every): iterations replayed per CUDA graph launch
    between host polls of the convergence word;
  - ensemble width s for a group of samples on one mesh (when the caller
    leaves it free): the width with the most member-iterations per second.
Each candidate is timed on the device (CUDA events around the CG SpMV
launches, or wall time of a fixed-iteration solve), and the winners are
cached in a JSON file keyed by GPU name and problem shape
(ENS_AUTOTUNE_CACHE, default ~/.cache/ens_autotune.json).
"""
import json
import os
import time

import paper_1511_03703_gb300 as E

FORMS = {"f64": 0, "df": E.CG_DF64, "split": E.CG_SPLIT64, "dfv": 0}  # dfv: ens_cg_df, pre-split values
CHECK_EVERY = (4, 8, 16, 32)
WIDTHS = (4, 8, 16, 32)
K1_CHUNKS = (1, 2, 4, 8)


def k1_chunk_choices(s):
    """Chunks of 32 rows per SpMV CTA that fit a 1024-thread CTA at width s."""
    threads_per_chunk = 32 * max(s // 2, 2)
    return tuple(c for c in K1_CHUNKS if c * threads_per_chunk <= 1024)


def k1_mapping_choices(s):
    """Every SpMV mapping at width s: the chunk counts and "defer"."""
    return k1_chunk_choices(s) + ("defer",)


def mapping_flags(mapping):
    """ens_cg flags of a tuned mapping {"form": ..., "k1_chunks": ...} (use
    values_df with the dfv form)."""
    return FORMS[mapping["form"]] | E.cg_k1_chunks(mapping.get("k1_chunks", 0))


def cache_path():
    return os.environ.get("ENS_AUTOTUNE_CACHE",
                          os.path.join(os.path.expanduser("~"), ".cache", "ens_autotune.json"))


def _load():
    try:
        with open(cache_path()) as f:
            return json.load(f)
    except (OSError, ValueError):
        return {}


def _store(db):
    path = cache_path()
    try:
        os.makedirs(os.path.dirname(path), exist_ok=True)
        tmp = path + f".tmp{os.getpid()}"
        with open(tmp, "w") as f:
            json.dump(db, f, indent=1, sort_keys=True)
        os.replace(tmp, path)
    except OSError:
        pass  # a read-only home: tuning still works, it is just not remembered


def _key(*parts):
    import torch
    return "|".join([torch.cuda.get_device_name()] + [str(p) for p in parts])


def _ensemble(mesh, s, seed=1004):
    import torch
    from paper_1511_03703_gb300 import inputs
    xs = inputs.kl_samples(seed, 0, s, mesh.M)
    dev = mesh.row_map.device
    vals, b = mesh.assemble(s, torch.from_numpy(inputs.ensemble_layout(xs)).to(dev))
    return vals, b


def time_spmv_mappings(mesh, s, iters=24, vals=None, b=None, candidates=tuple(FORMS), chunks=None):
    """Mean CG SpMV launch time (ms) of each (arithmetic form, chunks per CTA)
    on one ensemble: {(form, chunks): ms}.  chunks: the CTA mappings to try
    (default: every one that fits at width s)."""
    import torch
    if vals is None:
        vals, b = _ensemble(mesh, s)
    dev = vals.device
    work = torch.empty(E.cg_workspace_size(mesh.n, s), dtype=torch.uint8, device=dev)
    vdf = torch.empty(2 * vals.numel(), dtype=torch.float32, device=dev)
    E.convert_values(mesh.graph, s, vals, vdf, dtype=E.F64_DF)
    out = {}
    for name in candidates:
        for c in (chunks or k1_mapping_choices(s)):
            fl = FORMS[name] | E.cg_k1_chunks(c)
            vd = vdf if name == "dfv" else None
            x = torch.zeros(mesh.n * s, dtype=torch.float64, device=dev)
            E.cg(mesh.graph, s, vals, b, x, 0.0, 4, work, flags=fl, check_every=4, values_df=vd)
            x.zero_()
            _, _, _, st = E.cg(mesh.graph, s, vals, b, x, 0.0, iters, work,
                               flags=fl | E.CG_TIME_SPMV, check_every=iters, values_df=vd)
            out[(name, c)] = st.spmv_ms / max(st.spmv_launches, 1)
    return out


def time_spmv_forms(mesh, s, iters=24, vals=None, b=None, candidates=tuple(FORMS)):
    """Mean CG SpMV launch time (ms) of each arithmetic form on one ensemble,
    each at its fastest mapping."""
    t = time_spmv_mappings(mesh, s, iters, vals, b, candidates)
    return {f: min(ms for (g, _), ms in t.items() if g == f) for f in candidates}


def best_mapping(mesh, s, refresh=False, candidates=tuple(FORMS)):
    """Fastest (form, chunks per CTA) for (mesh, s) among `candidates`,
    cached: {"form": f, "k1_chunks": c, "spmv_ms": ms}."""
    db = _load()
    k = _key("mapping", mesh.N, mesh.M, s, ",".join(candidates))
    if not refresh and k in db:
        return db[k]
    t = time_spmv_mappings(mesh, s, candidates=candidates)
    (form, c), ms = min(t.items(), key=lambda kv: kv[1])
    db[k] = {"form": form, "k1_chunks": c, "spmv_ms": ms,
             "candidates_ms": {f"{f},{cc}": v for (f, cc), v in t.items()}}
    _store(db)
    return db[k]


def best_form(mesh, s, refresh=False, candidates=tuple(FORMS)):
    """Fastest SpMV form for (mesh, s) among `candidates` (at its best
    mapping), cached."""
    return best_mapping(mesh, s, refresh, candidates)["form"]


def best_check_every(batch, work, flags, iters=64, refresh=False, tag=""):
    """Graph length with the least wall time for `iters` iterations of a batch
    (tolerance 0: every candidate does the same work)."""
    import torch
    db = _load()
    k = _key("check_every", tag, flags)
    if not refresh and k in db:
        return db[k]["check_every"]
    res = {}
    for ce in CHECK_EVERY:
        batch.solve(0.0, ce, work, flags=flags | E.CG_GRAPH, check_every=ce)  # warm-up, capture
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        batch.solve(0.0, iters, work, flags=flags | E.CG_GRAPH, check_every=ce)
        torch.cuda.synchronize()
        res[ce] = time.perf_counter() - t0
    best = min(res, key=res.get)
    db[k] = {"check_every": best, "seconds": {str(c): v for c, v in res.items()}}
    _store(db)
    return best


def best_batch_k1(batch, work, flags, iters=48, refresh=False, tag=""):
    """CTA size of the batched SpMV (512, or 1024 threads with
    ENS_CG_BATCH_K1_WIDE) with the least wall time for `iters` iterations of
    the batch (tolerance 0); returns the flag to add (0 or the wide flag)."""
    import torch
    db = _load()
    k = _key("batch_k1", tag, flags)
    if not refresh and k in db:
        return db[k]["flag"]
    res = {}
    for wide in (0, E.CG_BATCH_K1_WIDE):
        fl = flags | wide | E.CG_GRAPH
        batch.solve(0.0, 8, work, flags=fl, check_every=8)  # warm-up, capture
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        batch.solve(0.0, iters, work, flags=fl, check_every=8)
        torch.cuda.synchronize()
        res[wide] = time.perf_counter() - t0
    best = min(res, key=res.get)
    db[k] = {"flag": best, "cta_threads": 1024 if best else 512,
             "seconds": {"512": res[0], "1024": res[E.CG_BATCH_K1_WIDE]}}
    _store(db)
    return best


def best_width(mesh, refresh=False):
    """Ensemble width with the most member-iterations per second of CG SpMV
    (each width at its own fastest form), for groups whose width is free."""
    db = _load()
    k = _key("width", mesh.N, mesh.M)
    if not refresh and k in db:
        return db[k]["width"], db[k]["form"]
    rates = {}
    for s in WIDTHS:
        t = time_spmv_forms(mesh, s)
        f = min(t, key=t.get)
        rates[s] = (s / t[f], f)
    s_best = max(rates, key=lambda v: rates[v][0])
    db[k] = {"width": s_best, "form": rates[s_best][1],
             "member_spmv_per_ms": {str(s): r for s, (r, _) in rates.items()}}
    _store(db)
    return s_best, rates[s_best][1]
