"""Edge cases, degenerate inputs and API behaviour of the CUDA path (GPU)."""
import numpy as np
import pytest

import oracle
from parity import coord_errors, knn_mismatches, report
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


def gpu(esom, w, chunk=None):
    with esom.Projector(w.d, w.L, w.k) as P:
        P.set_landmarks(torch.from_numpy(w.hi).cuda(), torch.from_numpy(w.lo).cuda())
        if chunk:
            P.set_landmark_chunk(chunk)
        X = torch.from_numpy(w.X).cuda()
        out = P.project(X, w.boost, w.adjust)
        idx, d2 = P.knn(X)
        torch.cuda.synchronize()
        assert P.device_status() == 0
        return out.cpu().numpy(), idx.cpu().numpy(), d2.cpu().numpy()


def against_oracle(w, out, idx, d2):
    o, ratio, branch = oracle.project(w.X, w.hi, w.lo, w.k, w.boost, w.adjust, diagnostics=True)
    oi, od = oracle.knn(w.X, w.hi, w.k)
    knn_mismatches(w.X, w.hi, idx, d2, oi, od)
    stats = coord_errors(out, o, ratio, w.extent)
    report(stats, w.name)
    return stats, branch


@pytest.mark.parametrize("d,L,k", [(4, 10, 3), (64, 50, 32), (8, 32, 32), (12, 7, 7),
                                   (24, 300, 2), (44, 90, 17), (20, 129, 9)])
def test_shapes(esom, d, L, k):
    rng = np.random.default_rng(d * 1000 + L + k)
    w = workloads.random_case(rng, 777, d, L, k, boost=1.3, adjust=1.0)
    out, idx, d2 = gpu(esom, w)
    against_oracle(w, out, idx, d2)


@pytest.mark.parametrize("adjust", [0.0, 0.5, 1.0, 2.0])
@pytest.mark.parametrize("boost", [0.5, 2.0])
def test_boost_adjust(esom, boost, adjust):
    rng = np.random.default_rng(11)
    w = workloads.random_case(rng, 1500, 16, 200, 12, boost=boost, adjust=adjust)
    out, idx, d2 = gpu(esom, w)
    against_oracle(w, out, idx, d2)


def test_k2_is_nearest_layout_point(esom):
    rng = np.random.default_rng(12)
    w = workloads.random_case(rng, 1000, 8, 40, 2)
    out, idx, _ = gpu(esom, w)
    assert np.array_equal(out, w.lo[idx[:, 0]])


def test_duplicate_and_coincident_landmarks(esom):
    """Pairs with L_u = L_v or l_u = l_v are skipped (their D or d is undefined)."""
    rng = np.random.default_rng(13)
    w = workloads.random_case(rng, 2000, 8, 60, 10)
    w.hi[30:40] = w.hi[0:10]          # duplicated high-dimensional landmarks
    w.lo[40:50] = w.lo[10:20]         # coincident 2-D landmarks
    out, idx, d2 = gpu(esom, w)
    against_oracle(w, out, idx, d2)


def test_collinear_layout_rank_one(esom):
    """All 2-D landmarks on a line: the rank-one solve on both sides."""
    rng = np.random.default_rng(14)
    w = workloads.random_case(rng, 2000, 8, 64, 10)
    a = rng.integers(0, 64, 64) / 8.0
    w.lo = np.stack([a, 0.5 * a - 2.0], 1).astype(np.float32)
    out, idx, d2 = gpu(esom, w)
    stats, branch = against_oracle(w, out, idx, d2)
    assert (branch == 1).all()


def test_exact_ties_lattice(esom):
    """Integer lattice points and landmarks: many exactly equal distances,
    resolved to the lower landmark index."""
    rng = np.random.default_rng(15)
    X = rng.integers(-3, 4, (3000, 4)).astype(np.float32)
    hi = rng.integers(-3, 4, (60, 4)).astype(np.float32)
    lo = rng.uniform(0, 10, (60, 2)).astype(np.float32)
    w = workloads.Workload("lattice", X, hi, lo, k=8, boost=1.0, adjust=1.0)
    with esom.Projector(4, 60, 8) as P:
        P.set_landmarks(torch.from_numpy(hi).cuda(), torch.from_numpy(lo).cuda())
        idx, d2 = P.knn(torch.from_numpy(X).cuda())
        torch.cuda.synchronize()
    oi, od = oracle.knn(X, hi, 8)
    assert np.array_equal(idx.cpu().numpy(), oi)          # exact integer arithmetic
    assert np.array_equal(d2.cpu().numpy().astype(np.float64), od)


def test_exact_plane_recovery(esom):
    """x = p when the landmarks are an exact similarity image of the plane."""
    rng = np.random.default_rng(16)
    d, g, k = 16, 256, 12
    cols = rng.choice(d, 4, replace=False)
    H = np.array([[1, 1, 1, 1], [1, -1, 1, -1]]) / 2.0
    Q = np.zeros((d, 2))
    Q[cols, :] = H.T
    lo = rng.integers(0, 128, (g, 2)) / 8.0
    hi = 2.0 * lo @ Q.T + rng.integers(-8, 8, d) / 4.0
    p = rng.integers(16, 240, (4000, 2)) / 16.0
    X = 2.0 * p @ Q.T + (hi[0] - 2.0 * lo[0] @ Q.T)
    w = workloads.Workload("plane", X.astype(np.float32), hi.astype(np.float32),
                           lo.astype(np.float32), k=k, boost=1.0, adjust=1.0)
    out, idx, d2 = gpu(esom, w)
    assert np.abs(out - p).max() <= 1e-4 * w.extent


def test_n_zero_and_errors(esom):
    w = workloads.mixture10_d8(n=100)
    with esom.Projector(w.d, w.L, w.k) as P:
        X = torch.from_numpy(w.X).cuda()
        st = esom.esom_project(P.h, X.data_ptr(), 100, X.data_ptr(), 1.0, 1.0, 0)
        assert st == esom.ESOM_ENOLANDMARKS
        P.set_landmarks(torch.from_numpy(w.hi).cuda(), torch.from_numpy(w.lo).cuda())
        out = torch.zeros((100, 2), device="cuda")
        assert esom.esom_project(P.h, X.data_ptr(), 0, out.data_ptr(), 1.0, 1.0, 0) == 0
        assert esom.esom_project(P.h, X.data_ptr() + 4, 99, out.data_ptr(), 1.0, 1.0, 0) \
            == esom.ESOM_EALIGN
        assert esom.esom_project(P.h, X.data_ptr(), 100, out.data_ptr(), 0.0, 1.0, 0) \
            == esom.ESOM_EINVAL
        assert esom.esom_project(P.h, X.data_ptr(), 100, out.data_ptr(), 1.0, -1.0, 0) \
            == esom.ESOM_EINVAL
        assert esom.esom_project(P.h, X.data_ptr(), -1, out.data_ptr(), 1.0, 1.0, 0) \
            == esom.ESOM_EINVAL
        torch.cuda.synchronize()
        assert (out == 0).all()      # nothing was launched


@pytest.mark.parametrize("plan", [0, 1, 2, 3])
def test_nan_input_no_fault(esom, plan):
    """NaN/Inf points give unspecified values but no fault, in every
    execution plan (fused, split, tensor-core); the context and later calls
    stay healthy."""
    w = workloads.mixture10_d8(n=3000)
    w.X[5] = np.nan
    w.X[6, 3] = np.inf
    with esom.Projector(w.d, w.L, w.k) as P:
        P.set_landmarks(torch.from_numpy(w.hi).cuda(), torch.from_numpy(w.lo).cuda())
        P.set_plan(plan)
        X = torch.from_numpy(w.X).cuda()
        P.project(X, 1.0, 1.0)
        P.knn(X)
        torch.cuda.synchronize()
        assert P.device_status() == 0
        good = np.ones(3000, bool)
        good[[5, 6]] = False
        out = P.project(X, 1.0, 1.0).cpu().numpy()
    o, ratio, _ = oracle.project(w.X[good], w.hi, w.lo, w.k, 1.0, 1.0, diagnostics=True)
    report(coord_errors(out[good], o, ratio, w.extent), f"non-finite rows, plan {plan}")


def test_deterministic_and_streams(esom):
    """Bitwise identical results across calls and on a side stream."""
    w = workloads.mixture30_d16(n=50_000)
    with esom.Projector(w.d, w.L, w.k) as P:
        P.set_landmarks(torch.from_numpy(w.hi).cuda(), torch.from_numpy(w.lo).cuda())
        X = torch.from_numpy(w.X).cuda()
        a = P.project(X, w.boost, w.adjust)
        s = torch.cuda.Stream()
        s.wait_stream(torch.cuda.current_stream())
        with torch.cuda.stream(s):
            b = P.project(X, w.boost, w.adjust)
        torch.cuda.synchronize()
        assert torch.equal(a, b)


def test_landmark_update_and_version(esom):
    w1 = workloads.mixture10_d8(seed=0, n=2000)
    w2 = workloads.mixture10_d8(seed=5, n=2000)
    with esom.Projector(w1.d, w1.L, w1.k) as P:
        assert esom.esom_landmark_version(P.h) == 0
        X = torch.from_numpy(w1.X).cuda()
        P.set_landmarks(torch.from_numpy(w1.hi).cuda(), torch.from_numpy(w1.lo).cuda())
        a = P.project(X).cpu().numpy()
        P.set_landmarks(torch.from_numpy(w2.hi).cuda(), torch.from_numpy(w2.lo).cuda())
        b = P.project(X).cpu().numpy()
        assert esom.esom_landmark_version(P.h) == 2
    o, ratio, _ = oracle.project(w1.X, w2.hi, w2.lo, w1.k, 1.0, 1.0, diagnostics=True)
    report(coord_errors(b, o, ratio, w2.extent), "landmark update")
    assert not np.allclose(a, b)


@pytest.mark.parametrize("pinned,n,plan", [(True, (1 << 20) * 2 + 1234, 0),
                                           (False, (1 << 20) * 2 + 1234, 0),
                                           (True, 1000, 0), (True, 77824 + 1, 0),
                                           (True, 2 * 77824 + 5, 0),
                                           (True, (1 << 19) + 2 * 77824 + 3, 0),
                                           (True, 58368 + 1, 2), (True, 2 * 58368 + 7, 3),
                                           (True, (1 << 20) + 12345, 2)])
def test_project_host_matches_device(esom, pinned, n, plan):
    """Host-buffer entry point (chunked H2D / kernel / D2H pipeline: a first
    and a last chunk of one k-NN wave, chunks of 2^19 between) gives the same
    bits as the device entry point; n spans one, two, three and several
    chunks."""
    w = workloads.mixture30_d16(n=n)
    with esom.Projector(w.d, w.L, w.k) as P:
        P.set_landmarks(torch.from_numpy(w.hi).cuda(), torch.from_numpy(w.lo).cuda())
        P.set_plan(plan)
        ref = P.project(torch.from_numpy(w.X).cuda(), w.boost, w.adjust).cpu()
        Xh = torch.from_numpy(w.X)
        if pinned:
            Xh = Xh.pin_memory()
        out = P.project_host(Xh, w.boost, w.adjust)
        torch.cuda.current_stream().synchronize()
        assert torch.equal(out, ref)


def test_ill_conditioned_points_every_path(esom):
    """With adjust = 2 on unstructured data about 4% of the points have a
    normal system with det/trace^2 < 1e-3, which FP32 sums cannot resolve
    (errors up to 35x the bound before); every execution plan, the batched
    launch and the no-alloc entry point list them and recompute them in
    FP64, one warp a point.  All return the same bits, within 1e-4 of the
    extent of the FP64 oracle, and the handle counts the recomputed points."""
    rng = np.random.default_rng(11)
    w = workloads.random_case(rng, 1500, 16, 200, 12, boost=2.0, adjust=2.0)
    X = torch.from_numpy(w.X).cuda()
    hi, lo = torch.from_numpy(w.hi).cuda(), torch.from_numpy(w.lo).cuda()
    outs = {}
    with esom.Projector(w.d, w.L, w.k) as P:
        P.set_landmarks(hi, lo)
        for plan, name in esom.PLAN_NAMES.items():
            P.set_plan(plan)
            P.stats(reset=True)
            outs[name] = P.project(X, w.boost, w.adjust).cpu().numpy()
            assert P.device_status() == 0
            assert P.stats()["refines"] > 0, name
        out_b = torch.empty((w.n, 2), device="cuda")
        P.set_plan(esom.ESOM_PLAN_FUSED)
        item = esom.BatchItem(P.h, X.data_ptr(), w.n, out_b.data_ptr(), w.boost, w.adjust)
        st, b = esom.esom_batch_create([item], False)
        assert st == 0
        assert esom.esom_batch_run(b, 0) == 0
        torch.cuda.synchronize()
        outs["batch"] = out_b.cpu().numpy()
        esom.esom_batch_destroy(b)
    out_n = torch.empty((w.n, 2), device="cuda")
    assert esom.esom_project_noalloc(X.data_ptr(), w.n, hi.data_ptr(), lo.data_ptr(), w.d, w.L,
                                     w.k, out_n.data_ptr(), w.boost, w.adjust, 0) == 0
    torch.cuda.synchronize()
    outs["noalloc"] = out_n.cpu().numpy()
    for name, o in outs.items():
        assert np.array_equal(o.view(np.uint32), outs["fused"].view(np.uint32)), name
    o, ratio, _ = oracle.project(w.X, w.hi, w.lo, w.k, w.boost, w.adjust, diagnostics=True)
    stats = coord_errors(outs["fused"], o, ratio, w.extent)
    report(stats, "ill-conditioned, every path")
    assert stats["ill_conditioned"] > 20
