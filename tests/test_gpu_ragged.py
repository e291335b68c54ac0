"""Ragged batches (items of different sizes in one plan) against the oracle and
against uniform plans of each item's size."""
import numpy as np
import pytest
import torch

import fp32_reference
import oracle.gfc_oracle as O
from paper_1902_00176_gb300 import gfc, synth

pytestmark = pytest.mark.gpu
DEV = torch.device("cuda:0")
REL_F32 = 1e-5


@pytest.fixture(autouse=True)
def _lib(gfc_lib):
    yield


def _rel(a, b):
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


def _items_small():
    return [(1, 37, 50), (3, 64, 96), (1, 20, 20), (2, 101, 33), (1, 64, 96), (3, 9, 140)]


def _inputs(items, seed=0):
    gxs, gys = [], []
    for i, (C, H, W) in enumerate(items):
        gx, gy = synth.ragged_item_gradients((C, H, W), item=i, seed=seed)
        gxs.append(torch.from_numpy(gx))
        gys.append(torch.from_numpy(gy))
    return gxs, gys


def test_ragged_matches_oracle_per_item():
    items = _items_small()
    gxs, gys = _inputs(items)
    rp = gfc.RaggedPlan(items, device=DEV)
    out = rp.unpack(rp.solve_from_gradient(rp.pack(gxs), rp.pack(gys)))
    torch.cuda.synchronize()
    for (C, H, W), gx, gy, o in zip(items, gxs, gys, out):
        M, N = gfc.padded_size(H, W)
        ref = O.solve_from_gradient_batch(gx.double().numpy(), gy.double().numpy(), M, N, 4)
        assert _rel(o.double().cpu().numpy(), ref) <= REL_F32, (C, H, W)
    rp.close()


def test_ragged_is_bitwise_equal_to_uniform_plans():
    """Each item of a ragged plan gives the same bits as a uniform plan of its size:
    items with register-resident row passes run as such plans (on internal streams),
    the others through the generic per-field passes."""
    items = _items_small()
    gxs, gys = _inputs(items, seed=1)
    rp = gfc.RaggedPlan(items, device=DEV)
    out = rp.unpack(rp.solve_from_gradient(rp.pack(gxs), rp.pack(gys)))
    for (C, H, W), gx, gy, o in zip(items, gxs, gys, out):
        p = gfc.Plan(H, W, C, 1, device=DEV)
        ref = p.solve_from_gradient(gx.view(1, C, H, W).to(DEV), gy.view(1, C, H, W).to(DEV))[0]
        assert torch.equal(o, ref), (C, H, W)
        p.close()
    rp.close()


def test_ragged_generic_items_match_uniform_generic_plans(monkeypatch):
    """With the register-resident passes switched off, every item runs the generic
    per-field passes and matches a generic uniform plan bit for bit."""
    items = _items_small()
    gxs, gys = _inputs(items, seed=1)
    monkeypatch.setenv("GFC_FORCE_GENERIC", "1")
    rp = gfc.RaggedPlan(items, device=DEV)
    out = rp.unpack(rp.solve_from_gradient(rp.pack(gxs), rp.pack(gys)))
    for (C, H, W), gx, gy, o in zip(items, gxs, gys, out):
        p = gfc.Plan(H, W, C, 1, device=DEV)
        ref = p.solve_from_gradient(gx.view(1, C, H, W).to(DEV), gy.view(1, C, H, W).to(DEV))[0]
        assert torch.equal(o, ref), (C, H, W)
        p.close()
    rp.close()


def test_ragged_workload_matches_uniform_plans_and_oracle():
    """The 64-item ragged workload (C in {1,3}, H, W in [128, 2048]) in one call:
    every item equals a uniform plan of its size bit for bit; three checked against
    the oracle in full."""
    items = synth.ragged_items()
    rp = gfc.RaggedPlan(items, device=DEV)
    gx, gy = rp.empty(), rp.empty()
    for i, (C, H, W) in enumerate(items):
        a, b = synth.ragged_item_gradients((C, H, W), item=i)
        o = rp.offsets[i]
        gx[o:o + C * H * W] = torch.from_numpy(a).reshape(-1).to(DEV)
        gy[o:o + C * H * W] = torch.from_numpy(b).reshape(-1).to(DEV)
    out = rp.solve_from_gradient(gx, gy)
    again = rp.solve_from_gradient(gx, gy)
    torch.cuda.synchronize()
    assert torch.equal(out, again)
    for i, (C, H, W) in enumerate(items):
        o = rp.offsets[i]
        p = gfc.Plan(H, W, C, 1, device=DEV)
        ref = p.solve_from_gradient(gx[o:o + C * H * W].view(1, C, H, W), gy[o:o + C * H * W].view(1, C, H, W))
        assert torch.equal(out[o:o + C * H * W], ref.reshape(-1)), items[i]
        p.close()
    for i in (0, 17, 63):
        C, H, W = items[i]
        o = rp.offsets[i]
        M, N = gfc.padded_size(H, W)
        ref = O.solve_from_gradient(gx[o:o + H * W].view(H, W).double().cpu().numpy(),
                                    gy[o:o + H * W].view(H, W).double().cpu().numpy(), M, N, 4)
        got = out[o:o + H * W].view(H, W).double().cpu().numpy()
        assert _rel(got, ref) <= REL_F32, items[i]
    rp.close()


def test_ragged_laplacian_and_adjoint_modes():
    items = [(1, 30, 45), (2, 17, 64), (1, 64, 20), (2, 150, 300), (1, 40, 700)]
    rng = np.random.default_rng(3)
    laps = [torch.from_numpy(rng.standard_normal((C, H, W)).astype(np.float32) * 0.01) for (C, H, W) in items]
    rp = gfc.RaggedPlan(items, device=DEV)
    out = rp.unpack(rp.solve_from_laplacian(rp.pack(laps)))
    bx, by = rp.backward(rp.pack(laps))
    bx, by = rp.unpack(bx), rp.unpack(by)
    torch.cuda.synchronize()
    for (C, H, W), lap, o, gx_, gy_ in zip(items, laps, out, bx, by):
        M, N = gfc.padded_size(H, W)
        ref = O.solve_from_laplacian_batch(lap.double().numpy(), M, N, 4)
        rx, ry = O.backward_batch(lap.double().numpy(), M, N, 4)
        # white-noise inputs: the FP32 bar is 3x a plain torch FP32 evaluation's error
        for c in range(C):
            l64 = lap[c].double().numpy()
            t_u = fp32_reference.torch_fp32_laplacian_solve(l64, M, N, 4, DEV)
            t_x, t_y = fp32_reference.torch_fp32_adjoint(l64, M, N, 4, DEV)
            assert _rel(o[c].double().cpu().numpy(), ref[c]) <= max(REL_F32, 3.0 * _rel(t_u, ref[c])), (C, H, W)
            assert _rel(gx_[c].double().cpu().numpy(), rx[c]) <= max(REL_F32, 3.0 * _rel(t_x, rx[c])), (C, H, W)
            assert _rel(gy_[c].double().cpu().numpy(), ry[c]) <= max(REL_F32, 3.0 * _rel(t_y, ry[c])), (C, H, W)
    rp.close()


def test_captured_graphs_replay_the_same_solve():
    items = _items_small()
    gxs, gys = _inputs(items, seed=5)
    rp = gfc.RaggedPlan(items, device=DEV)
    gx, gy = rp.pack(gxs), rp.pack(gys)
    ref = rp.solve_from_gradient(gx, gy).clone()
    out = rp.empty()
    g = gfc.Graph(rp, "gradient", gx, gy, out)
    g.launch()
    torch.cuda.synchronize()
    assert torch.equal(out, ref)
    gx2 = gx * 2.0
    gx.copy_(gx2)  # new contents, same buffers
    g.launch()
    torch.cuda.synchronize()
    assert torch.equal(out, rp.solve_from_gradient(gx, gy))
    g.close()
    # uniform plan, fast path, backward op
    p = gfc.Plan(801, 1200, 1, 2, device=DEV)
    go = torch.randn((2, 1, 801, 1200), device=DEV)
    bx, by = torch.empty_like(go), torch.empty_like(go)
    g2 = gfc.Graph(p, "backward", go, None, bx, by)
    g2.launch()
    rx, ry = p.backward(go)
    torch.cuda.synchronize()
    assert torch.equal(bx, rx) and torch.equal(by, ry)
    g2.close()
    p.close()
    rp.close()
