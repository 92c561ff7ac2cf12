"""Tensor-core screening (ESOM_SCREEN_TF32) against the plain FP32 path and
the oracle (GPU).

The screened path only changes how candidates are found: the listed ones are
re-ranked with the same exact FP32 distances and certified, so neighbours,
distances and coordinates must equal the FP32 path's bit for bit; the rate of
certificate failures (exact rescans) is reported and bounded."""
import json

import numpy as np
import pytest

from paper_2201_00701_gb300 import workloads
from test_gpu_parity import check

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def esom():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2201_00701_gb300 import binding
    binding.load(build_if_missing=True)
    return binding


def run_mode(esom, w, mode, X=None):
    X = torch.from_numpy(w.X).cuda() if X is None else X
    with esom.Projector(w.d, w.L, w.k) as P:
        P.set_landmarks(torch.from_numpy(w.hi).cuda(), torch.from_numpy(w.lo).cuda())
        P.set_screening(mode)
        out = torch.full((X.shape[0], 2), float("nan"), device="cuda")
        P.project(X, w.boost, w.adjust, out=out)
        idx, d2 = P.knn(X)
        torch.cuda.synchronize()
        assert P.device_status() == 0
        cfg = P.config()
        cfg["stats"] = P.stats()
    return out.cpu().numpy(), idx.cpu().numpy(), d2.cpu().numpy(), cfg


def same_as_fp32(esom, w, label, max_rescans=0.02, mode=None):
    mode = esom.ESOM_SCREEN_TF32 if mode is None else mode
    ref = run_mode(esom, w, esom.ESOM_SCREEN_FP32)
    got = run_mode(esom, w, mode)
    cfg = got[3]
    assert cfg["screening"] == mode and ref[3]["screening"] == 0
    frac = cfg["stats"]["rescans"] / max(cfg["stats"]["points"], 1)
    print("TC", json.dumps({"label": label, "mode": {1: "tf32", 2: "bf16"}[mode],
                            "n": w.n, "d": w.d, "L": w.L, "k": w.k,
                            "rescan_fraction": frac, "blocks_per_sm": cfg["blocks_per_sm"],
                            "shared_bytes": cfg["shared_bytes"]}))
    assert np.array_equal(got[1], ref[1]), "k-NN indices differ from the FP32 path"
    assert np.array_equal(got[2].view(np.uint32), ref[2].view(np.uint32)), "distances differ"
    assert np.array_equal(got[0].view(np.uint32), ref[0].view(np.uint32)), "coordinates differ"
    assert frac <= max_rescans
    return got


@pytest.mark.parametrize("n", [1, 127, 128, 129, 20_000 + 77, (1 << 20) + 1000])
def test_mixture30_d16_equals_fp32(esom, n):
    """Tile edges, a ragged tail, and two k-NN passes (n above 2^20)."""
    w = workloads.mixture30_d16(n=n)
    same_as_fp32(esom, w, f"mixture30_d16 n={n}")


def test_mixture10_d8_equals_fp32_and_oracle(esom):
    w = workloads.mixture10_d8()
    out, idx, d2, cfg = same_as_fp32(esom, w, "mixture10_d8")
    check(w, out, idx, d2, label="mixture10_d8 tf32", cfg=cfg, max_rescans=0.02)


def test_student50_d32_equals_fp32(esom):
    """d = 32, L = 4096 (64 chunks), k = 30 on 300,000 points."""
    w = workloads.student50_d32(n=300_000)
    out, idx, d2, cfg = same_as_fp32(esom, w, "student50_d32 n=3e5", max_rescans=0.05)
    rows = np.random.default_rng(3).choice(w.n, 1500, replace=False)
    check(w, out, idx, d2, rows=rows, label="student50_d32 tf32 sampled", cfg=cfg,
          max_rescans=0.05)


@pytest.mark.parametrize("name", ["uniform_d16", "uniform_d32"])
def test_paper_shape_equals_fp32(esom, name):
    same_as_fp32(esom, workloads.make(name, n=50_000), name)


@pytest.mark.parametrize("i", [1, 4, 5, 9, 17])
def test_batch_members_equal_fp32(esom, i):
    """Members of the 64-dataset mix: d in {8, 16, 32, 48}, L up to 2500,
    k up to 30."""
    p = workloads.batch64()[i]
    w = workloads.batch_member(p, n=min(p["n"], 30_000))
    # member 4 (d=48, L=2500, k=10: dense clusters, 6 spare list entries) rescans ~25%
    same_as_fp32(esom, w, f"batch64[{i}] d={w.d} L={w.L} k={w.k}", max_rescans=0.3)


@pytest.mark.parametrize("d,L,k", [(4, 300, 10), (12, 70, 8), (20, 129, 20), (28, 64, 32),
                                   (36, 500, 16), (44, 65, 5), (52, 200, 12), (60, 1000, 30),
                                   (64, 333, 20), (16, 7, 3), (8, 2, 2), (24, 1, 1)])
def test_shapes_equal_fp32(esom, d, L, k):
    """Every D-instantiation family, ragged chunks, L below one chunk."""
    if k > L:
        k = L
    if k < 2:
        pytest.skip("k >= 2")
    r = np.random.default_rng(d * 1000 + L)
    w = workloads.random_case(r, 3000, d, L, k, boost=1.5, adjust=0.5)
    same_as_fp32(esom, w, f"random d={d} L={L} k={k}", max_rescans=0.2)


def test_far_from_origin_is_still_exact(esom):
    """Points and landmarks shifted far from the origin: the screening bound
    grows with |x| max|l|, so more points are rescanned, but results stay
    the FP32 path's."""
    r = np.random.default_rng(11)
    w = workloads.random_case(r, 4000, 16, 512, 12)
    w.X = (w.X + 200.0).astype(np.float32)
    w.hi = (w.hi + 200.0).astype(np.float32)
    same_as_fp32(esom, w, "shifted by 200", max_rescans=1.0)


@pytest.mark.parametrize("n,L,k", [(200, 512, 12), (300, 70, 20), (5, 1000, 32), (2000, 300, 8)])
def test_rescan_modes(esom, n, L, k):
    """Shifted data: every point fails its certificate.  Up to one failed
    point per rescan block (n <= 304 here) the block-per-point rescan runs,
    above it the warp-per-point one; both give the FP32 path's bits, also
    with fewer landmarks than threads in a block (L = 70)."""
    r = np.random.default_rng(n + L)
    w = workloads.random_case(r, n, 16, L, k)
    w.X = (w.X + 200.0).astype(np.float32)
    w.hi = (w.hi + 200.0).astype(np.float32)
    for mode in (esom.ESOM_SCREEN_TF32, esom.ESOM_SCREEN_BF16):
        same_as_fp32(esom, w, f"rescan n={n} L={L} k={k}", max_rescans=1.0, mode=mode)


def test_landmark_update_rebuilds_images(esom):
    """set_landmarks after switching to TF32 rebuilds the chunk images."""
    w1 = workloads.mixture30_d16(n=5000)
    w2 = workloads.mixture30_d16(seed=1, n=5000)
    X = torch.from_numpy(w1.X).cuda()
    with esom.Projector(w1.d, w1.L, w1.k) as P:
        P.set_landmarks(torch.from_numpy(w1.hi).cuda(), torch.from_numpy(w1.lo).cuda())
        P.set_screening(esom.ESOM_SCREEN_TF32)
        P.project(X, w1.boost, w1.adjust)
        P.set_landmarks(torch.from_numpy(w2.hi).cuda(), torch.from_numpy(w2.lo).cuda())
        got = P.project(X, w1.boost, w1.adjust).cpu().numpy()
        P.set_screening(esom.ESOM_SCREEN_FP32)
        ref = P.project(X, w1.boost, w1.adjust).cpu().numpy()
        assert P.device_status() == 0
    assert np.array_equal(got.view(np.uint32), ref.view(np.uint32))


def test_screening_before_landmarks_and_errors(esom):
    w = workloads.mixture10_d8(n=3000)
    X = torch.from_numpy(w.X).cuda()
    with esom.Projector(w.d, w.L, w.k) as P:
        assert esom.esom_set_screening(P.h, 7, 0) == esom.ESOM_EINVAL
        P.set_screening(esom.ESOM_SCREEN_TF32)  # images built by set_landmarks
        P.set_landmarks(torch.from_numpy(w.hi).cuda(), torch.from_numpy(w.lo).cuda())
        got = P.project(X, w.boost, w.adjust).cpu().numpy()
        assert P.project(X[:0], w.boost, w.adjust).shape == (0, 2)
        assert P.config()["threads_per_block"] == 160
    ref = run_mode(esom, w, esom.ESOM_SCREEN_FP32)[0]
    assert np.array_equal(got.view(np.uint32), ref.view(np.uint32))


def test_side_stream_and_repeat(esom):
    """Same bits on a side stream and on repeated launches."""
    w = workloads.mixture30_d16(n=40_000)
    X = torch.from_numpy(w.X).cuda()
    with esom.Projector(w.d, w.L, w.k) as P:
        P.set_landmarks(torch.from_numpy(w.hi).cuda(), torch.from_numpy(w.lo).cuda())
        P.set_screening(esom.ESOM_SCREEN_TF32)
        a = P.project(X, w.boost, w.adjust)
        s = torch.cuda.Stream()
        s.wait_stream(torch.cuda.current_stream())
        with torch.cuda.stream(s):
            b = P.project(X, w.boost, w.adjust)
        s.synchronize()
        c = P.project(X, w.boost, w.adjust)
        torch.cuda.synchronize()
    assert torch.equal(a, b) and torch.equal(a, c)


@pytest.mark.parametrize("case", ["mixture30_d16", "mixture10_d8", "uniform_d32", "chunked",
                                  "batch4", "shifted"])
def test_split_equals_fused(esom, case):
    """FP32 screening as two kernels (k-NN, then projection from the
    neighbours) gives the fused kernel's bits, also across pass boundaries
    (n above 2^20) and with streamed landmark chunks."""
    chunk = None
    if case == "mixture30_d16":
        w = workloads.mixture30_d16(n=(1 << 20) + 70_000)
    elif case == "mixture10_d8":
        w = workloads.mixture10_d8()
    elif case == "uniform_d32":
        w = workloads.make("uniform_d32", n=50_000)
    elif case == "chunked":
        w = workloads.mixture30_d16(n=30_000)
        chunk = 200
    elif case == "shifted":  # every point fails its certificate: deferred rescans
        w = workloads.random_case(np.random.default_rng(11), 4000, 16, 512, 12)
        w.X = (w.X + 200.0).astype(np.float32)
        w.hi = (w.hi + 200.0).astype(np.float32)
    else:
        p = workloads.batch64()[4]
        w = workloads.batch_member(p, n=min(p["n"], 20_000))
    X = torch.from_numpy(w.X).cuda()
    outs = []
    with esom.Projector(w.d, w.L, w.k) as P:
        P.set_landmarks(torch.from_numpy(w.hi).cuda(), torch.from_numpy(w.lo).cuda())
        if chunk:
            P.set_landmark_chunk(chunk)
        for split in (False, True):
            P.set_split(split)
            outs.append(P.project(X, w.boost, w.adjust).cpu().numpy())
        torch.cuda.synchronize()
        assert P.device_status() == 0
    assert np.array_equal(outs[0].view(np.uint32), outs[1].view(np.uint32))


@pytest.mark.parametrize("name", ["mixture30_d16", "uniform_d16"])
def test_tune_picks_a_plan_with_the_same_bits(esom, name):
    """esom_tune times the fused, split, TF32 and BF16 plans on the points,
    keeps the fastest, and every plan gives the same coordinates."""
    w = workloads.make(name, n=200_000)
    X = torch.from_numpy(w.X).cuda()
    with esom.Projector(w.d, w.L, w.k) as P:
        P.set_landmarks(torch.from_numpy(w.hi).cuda(), torch.from_numpy(w.lo).cuda())
        outs = {}
        for plan in esom.PLAN_NAMES:
            P.set_plan(plan)
            assert P.config()["plan"] == plan
            outs[plan] = P.project(X, w.boost, w.adjust).cpu().numpy()
        chosen = P.tune(X, w.boost, w.adjust)
        assert chosen in outs and P.config()["plan"] == chosen
        got = P.project(X, w.boost, w.adjust).cpu().numpy()
        print("TUNE", name, esom.PLAN_NAMES[chosen])
    for o in outs.values():
        assert np.array_equal(o.view(np.uint32), got.view(np.uint32))



@pytest.mark.parametrize("d,L,k", [(4, 300, 10), (12, 70, 8), (16, 1024, 20), (20, 129, 20),
                                   (28, 64, 32), (32, 500, 16), (36, 500, 16), (52, 200, 12),
                                   (64, 333, 20), (8, 2, 2)])
def test_bf16_shapes_equal_fp32(esom, d, L, k):
    """BF16 screening (half the operand bytes, 64-byte rows up to d = 32)
    gives the FP32 path's bits too; its larger error bound only shows in the
    rescan rate."""
    r = np.random.default_rng(d * 1000 + L + 7)
    w = workloads.random_case(r, 3000, d, L, k, boost=1.5, adjust=0.5)
    same_as_fp32(esom, w, f"bf16 random d={d} L={L} k={k}", max_rescans=0.5,
                 mode=esom.ESOM_SCREEN_BF16)


@pytest.mark.parametrize("name", ["mixture30_d16", "student50_d32"])
def test_bf16_named_equal_fp32(esom, name):
    w = workloads.make(name, n=100_000)
    same_as_fp32(esom, w, f"bf16 {name}", max_rescans=0.2, mode=esom.ESOM_SCREEN_BF16)
