"""The autotuner on the GPU: it keeps a working configuration of the same
problem (results unchanged up to the column solver's FP32 rounding), records its
choice in the cache, and a later plan of the same problem reads it back."""
import numpy as np
import pytest
import torch

from paper_1902_00176_gb300 import gfc, synth

pytestmark = pytest.mark.gpu
DEV = torch.device("cuda:0")


@pytest.fixture(autouse=True)
def _lib(gfc_lib):
    yield


def _rel(a, b):
    a, b = a.double().cpu().numpy(), b.double().cpu().numpy()
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


def test_autotune_uniform_plan_and_cache(tmp_path):
    B, H, W = 12, 801, 1200
    gx, gy = synth.perturbed_gradient_batch(batch=B, H=H, W=W, seed=9300)
    tx, ty = torch.from_numpy(gx).to(DEV), torch.from_numpy(gy).to(DEV)
    p = gfc.Plan(H, W, 1, B, device=DEV)
    before = p.solve_from_gradient(tx, ty)
    cache = str(tmp_path / "tune.txt")
    r = p.autotune(cache)
    assert r["from_cache"] == 0 and r["candidates"] >= 2 and r["ms"] > 0
    assert r["column_solver"] in (0, 1) and r["streams"] in (1, 2, 3, 4) and r["block_items"] in (0, 1)
    after = p.solve_from_gradient(tx, ty)
    assert _rel(after, before) <= 2e-6
    assert gfc.tune_cache_get(cache, p.tune_key()) is not None
    q = gfc.Plan(H, W, 1, B, device=DEV)
    r2 = q.autotune(cache)
    assert r2["from_cache"] == 1 and r2["column_solver"] == r["column_solver"] and r2["chunk"] == r["chunk"]
    assert r2["streams"] == r["streams"] and r2["block_items"] == r["block_items"]
    assert torch.equal(q.solve_from_gradient(tx, ty), after)
    p.close()
    q.close()


def test_autotune_ragged_plan_keeps_its_results(tmp_path):
    items = [(3, 300, 500), (1, 1000, 700), (1, 150, 1800), (3, 640, 480), (1, 100, 90)]
    rp = gfc.RaggedPlan(items, device=DEV)
    gxs, gys = [], []
    for i, (C, H, W) in enumerate(items):
        a, b = synth.ragged_item_gradients((C, H, W), item=i, seed=9400)
        gxs.append(torch.from_numpy(a))
        gys.append(torch.from_numpy(b))
    gx, gy = rp.pack(gxs), rp.pack(gys)
    before = rp.solve_from_gradient(gx, gy).clone()
    cache = str(tmp_path / "tune.txt")
    r = rp.autotune(cache)
    assert r["rag_streams"] in (1, 2, 4, 8) and r["candidates"] >= 2
    assert torch.equal(rp.solve_from_gradient(gx, gy), before)
    rp2 = gfc.RaggedPlan(items, device=DEV)
    r2 = rp2.autotune(cache)
    assert r2["from_cache"] == 1 and r2["rag_streams"] == r["rag_streams"]
    assert torch.equal(rp2.solve_from_gradient(gx, gy), before)
    rp.close()
    rp2.close()


@pytest.mark.parametrize("H,W,B", [(801, 1200, 7), (256, 256, 40)])
def test_block_per_item_grids_give_the_same_bits(H, W, B):
    """One block per item runs the same per-item arithmetic as the persistent grids:
    results are bitwise equal, whole batch and in chunks over streams."""
    gx, gy = synth.perturbed_gradient_batch(batch=B, H=H, W=W, seed=9500 + H)
    tx, ty = torch.from_numpy(gx).to(DEV), torch.from_numpy(gy).to(DEV)
    ref = gfc.Plan(H, W, 1, B, device=DEV)
    want = ref.solve_from_gradient(tx, ty)
    for chunk, streams in ((0, 1), (3, 2)):
        p = gfc.Plan(H, W, 1, B, device=DEV, chunk=chunk, streams=streams, block_items=True)
        assert torch.equal(p.solve_from_gradient(tx, ty), want), (chunk, streams)
        p.close()
    ref.close()
