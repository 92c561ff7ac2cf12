"""Batched projection (one persistent launch per (d, k-capacity) group,
cost-balanced tile ranges, optional autotuning and CUDA-graph replay)
against the single-dataset path and the oracle (GPU)."""
import json

import numpy as np
import pytest

import oracle
from parity import coord_errors, report
from paper_2201_00701_gb300 import workloads

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def esom():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2201_00701_gb300 import binding
    binding.load(build_if_missing=True)
    return binding


def _members(count, n_cap):
    params = workloads.batch64()[:count]
    return [workloads.batch_member(p, n=min(p["n"], n_cap)) for p in params]


@pytest.mark.parametrize("autotune", [False, True])
def test_batch_matches_single_launches(esom, autotune):
    """Every dataset's coordinates from the batch equal (bitwise) those of
    its own esom_project launch; plain run and graph replay agree."""
    ws = _members(12, 20_000)
    handles, items, outs, refs, keep = [], [], [], [], []
    for w in ws:
        P = esom.Projector(w.d, w.L, w.k)
        hi, lo = torch.from_numpy(w.hi).cuda(), torch.from_numpy(w.lo).cuda()
        P.set_landmarks(hi, lo)
        X = torch.from_numpy(w.X).cuda()
        out = torch.full((w.n, 2), float("nan"), device="cuda")
        refs.append(P.project(X, w.boost, w.adjust))
        items.append(esom.BatchItem(P.h, X.data_ptr(), w.n, out.data_ptr(), w.boost, w.adjust))
        handles.append(P)
        outs.append(out)
        keep.append((X, hi, lo))
    st, b = esom.esom_batch_create(items, autotune)
    assert st == 0, esom.esom_last_error()
    plan = json.loads(esom.esom_batch_plan(b))
    print("BATCH_PLAN", json.dumps(plan))
    assert sum(g["datasets"] for g in plan["groups"]) == len(ws)
    assert esom.esom_batch_run(b, torch.cuda.current_stream().cuda_stream) == 0
    torch.cuda.synchronize()
    for o, r in zip(outs, refs):
        assert torch.equal(o, r)
    for o in outs:
        o.fill_(float("nan"))
    assert esom.esom_batch_run_graph(b, torch.cuda.current_stream().cuda_stream) == 0
    assert esom.esom_batch_run_graph(b, torch.cuda.current_stream().cuda_stream) == 0
    torch.cuda.synchronize()
    for o, r in zip(outs, refs):
        assert torch.equal(o, r)
    esom.esom_batch_destroy(b)
    for P in handles:
        P.close()


def test_batch_against_oracle(esom):
    ws = _members(6, 3000)
    items, outs, keep, handles = [], [], [], []
    for w in ws:
        P = esom.Projector(w.d, w.L, w.k)
        hi, lo = torch.from_numpy(w.hi).cuda(), torch.from_numpy(w.lo).cuda()
        P.set_landmarks(hi, lo)
        X = torch.from_numpy(w.X).cuda()
        out = torch.empty((w.n, 2), device="cuda")
        items.append(esom.BatchItem(P.h, X.data_ptr(), w.n, out.data_ptr(), w.boost, w.adjust))
        outs.append(out)
        keep.append((X, hi, lo))
        handles.append(P)
    st, b = esom.esom_batch_create(items, False)
    assert st == 0
    assert esom.esom_batch_run(b, 0) == 0
    torch.cuda.synchronize()
    for w, out in zip(ws, outs):
        ref, ratio, _ = oracle.project(w.X, w.hi, w.lo, w.k, w.boost, w.adjust, diagnostics=True)
        report(coord_errors(out.cpu().numpy(), ref, ratio, w.extent), w.name)
    esom.esom_batch_destroy(b)
    for P in handles:
        P.close()
