"""Batched CG (one launch per CG phase for a mix of meshes and ensemble sizes)
against separate ens_cg solves of the same ensembles, and against the oracle.

The batched kernels run the same per-chunk arithmetic as the single-ensemble
kernels, so every member must come out bitwise identical."""
import numpy as np
import pytest

import oracle as O
import paper_1511_03703_gb300 as E
from paper_1511_03703_gb300 import inputs
from helpers import gpu, oracle_members, to_dev, to_np

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def torch():
    import torch as T
    assert T.cuda.is_available()
    E.lib()
    return T


def make_items(torch, spec, seed=500):
    items, meta = [], []
    meshes = {}
    for k, (N, s) in enumerate(spec):
        mesh = meshes.setdefault(N, E.Mesh(N, 10))
        xs = inputs.kl_samples(seed + k, 0, s, 10)
        vals, b = mesh.assemble(s, to_dev(inputs.ensemble_layout(xs)))
        x = torch.zeros(mesh.n * s, dtype=torch.float64, device=gpu())
        items.append((mesh.graph, s, vals, b, x))
        meta.append((mesh, xs))
    return items, meta


SPEC = [(5, 4), (9, 32), (7, 1), (12, 8), (9, 16), (5, 32), (3, 4)]


@pytest.mark.parametrize("flags", [0, E.CG_SPLIT64, E.CG_DF64 | E.CG_GRAPH, E.CG_GRAPH,
                                   E.CG_BATCH_K1_WIDE, E.CG_SPLIT64 | E.CG_BATCH_K1_WIDE | E.CG_GRAPH])
def test_batched_equals_separate_solves_bitwise(torch, flags):
    items, meta = make_items(torch, SPEC)
    batch = E.Batch(items)
    work = torch.empty(batch.workspace_size(), dtype=torch.uint8, device=gpu())
    it_b, rr_b, st_b, stats = batch.solve(1e-9, 2000, work, flags=flags, check_every=4)
    assert stats.kernel_launches > 0
    for i, (graph, s, vals, b, x) in enumerate(items):
        assert st_b[i] == [0] * s
        x2 = torch.zeros_like(x)
        w2 = torch.empty(E.cg_workspace_size(graph.num_rows, s), dtype=torch.uint8, device=gpu())
        it, rr, st, _ = E.cg(graph, s, vals, b, x2, 1e-9, 2000, w2, flags=flags & ~(E.CG_GRAPH | E.CG_BATCH_K1_WIDE))
        assert it == it_b[i] and rr == rr_b[i]
        assert torch.equal(x, x2), i


@pytest.mark.parametrize("flags", [0, E.CG_GRAPH])
def test_batched_presplit_equals_separate_cg_df_bitwise(torch, flags):
    """Items with pre-split values: the batch runs the ens_cg_df arithmetic."""
    items, meta = make_items(torch, SPEC, seed=540)
    pitems = []
    for graph, s, vals, b, x in items:
        vdf = torch.empty(2 * vals.numel(), dtype=torch.float32, device=gpu())
        E.convert_values(graph, s, vals, vdf, dtype=E.F64_DF)
        pitems.append((graph, s, vals, b, x, vdf))
    batch = E.Batch(pitems)
    work = torch.empty(batch.workspace_size(), dtype=torch.uint8, device=gpu())
    it_b, rr_b, st_b, _ = batch.solve(1e-9, 2000, work, flags=flags, check_every=4)
    for i, (graph, s, vals, b, x, vdf) in enumerate(pitems):
        assert st_b[i] == [0] * s
        x2 = torch.zeros_like(x)
        w2 = torch.empty(E.cg_workspace_size(graph.num_rows, s), dtype=torch.uint8, device=gpu())
        it, rr, st, _ = E.cg(graph, s, vals, b, x2, 1e-9, 2000, w2, values_df=vdf)
        assert it == it_b[i] and rr == rr_b[i]
        assert torch.equal(x, x2), i
    # every item or none; no second arithmetic flag
    with pytest.raises(E.EnsError) as ei:
        E.Batch(pitems[:2] + [items[2]]).workspace_size()
    assert ei.value.code == 1
    with pytest.raises(E.EnsError) as ei:
        batch.solve(1e-9, 10, work, flags=E.CG_DF64)
    assert ei.value.code == 1


def test_batched_matches_oracle(torch):
    items, meta = make_items(torch, [(6, 4), (10, 8)], seed=610)
    batch = E.Batch(items)
    work = torch.empty(batch.workspace_size(), dtype=torch.uint8, device=gpu())
    it_b, rr_b, st_b, _ = batch.solve(1e-10, 2000, work, flags=E.CG_SPLIT64, check_every=8)
    for i, (graph, s, vals, b, x) in enumerate(items):
        mesh, xs = meta[i]
        rm, col, ov, ob = oracle_members(mesh.N, 10, xs)
        X = to_np(x).reshape(-1, s)
        for e in range(s):
            xo, ito, _, sto = O.cg(rm, col, ov[e], ob[e], tol=1e-12)
            assert np.linalg.norm(X[:, e] - xo) <= 1e-8 * np.linalg.norm(xo)


def test_batched_argument_errors(torch):
    items, _ = make_items(torch, [(4, 4)])
    graph, s, vals, b, x = items[0]
    bad = E.Batch([(graph, 4, vals, b, x)])
    small = torch.empty(16, dtype=torch.uint8, device=gpu())
    with pytest.raises(E.EnsError) as ei:
        bad.solve(1e-8, 10, small)
    assert ei.value.code == 9
    bad2 = E.Batch([(graph, 3, vals, b, x)])
    with pytest.raises(E.EnsError) as ei:
        bad2.workspace_size()
    assert ei.value.code == 2


def test_autotuner_picks_and_caches(torch, tmp_path, monkeypatch):
    from paper_1511_03703_gb300 import autotune
    monkeypatch.setenv("ENS_AUTOTUNE_CACHE", str(tmp_path / "tune.json"))
    mesh = E.Mesh(12, 10)
    form = autotune.best_form(mesh, 8)
    assert form in autotune.FORMS
    assert autotune.best_form(mesh, 8) == form          # served from the cache
    import json
    db = json.loads((tmp_path / "tune.json").read_text())
    key = next(k for k in db if "|mapping|12|10|8|" in k)
    assert db[key]["form"] == form and db[key]["k1_chunks"] in autotune.k1_mapping_choices(8)
    s, f = autotune.best_width(mesh)
    assert s in autotune.WIDTHS and f in autotune.FORMS
    items, _ = make_items(torch, [(6, 4), (8, 8)])
    batch = E.Batch(items)
    work = torch.empty(batch.workspace_size(), dtype=torch.uint8, device=gpu())
    assert autotune.best_check_every(batch, work, 0, iters=16, tag="t") in autotune.CHECK_EVERY
