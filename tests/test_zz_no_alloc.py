"""esom_project_noalloc: the projection for callers that cannot allocate
device memory (a pool allocator owns all of it, or a frame loop must avoid
cudaMalloc's device-wide synchronisation).  Its scratch is a fixed device
array inside the library; this file checks, through the C ABI, that it gives
the same coordinates as the handle-based esom_project on consecutive calls
that reuse that scratch, and that it refuses landmark sets too large for it.
Kept in a file of its own that pytest collects last (GPU)."""
import numpy as np
import pytest

from parity import COORD_TOL
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


def _noalloc(esom, w, X, hi, lo):
    out = torch.full((w.n, 2), float("nan"), device="cuda")
    st = esom.esom_project_noalloc(X.data_ptr(), w.n, hi.data_ptr(), lo.data_ptr(), w.d, w.L,
                                   w.k, out.data_ptr(), w.boost, w.adjust,
                                   torch.cuda.current_stream().cuda_stream)
    assert st == esom.ESOM_OK, esom.esom_last_error()
    return out


def test_noalloc_matches_handle_path_on_consecutive_calls(esom):
    # Three calls in a row share the one scratch array: two landmark sets of
    # the same shape, then a different shape.
    cases = [workloads.mixture30_d16(seed=0, n=60_000),
             workloads.mixture30_d16(seed=3, n=40_000),
             workloads.mixture10_d8(seed=1, n=30_000)]
    for w in cases:
        X = torch.from_numpy(w.X).cuda()
        hi = torch.from_numpy(w.hi).cuda()
        lo = torch.from_numpy(w.lo).cuda()
        got = _noalloc(esom, w, X, hi, lo)
        with esom.Projector(w.d, w.L, w.k) as P:
            P.set_landmarks(hi, lo)
            ref = P.project(X, w.boost, w.adjust)
            torch.cuda.synchronize()
        got, ref = got.cpu().numpy(), ref.cpu().numpy()
        assert np.isfinite(got).all()
        err = np.abs(got.astype(np.float64) - ref).max()
        assert err <= COORD_TOL * w.extent, f"{w.name}: {err:.3e}"


def test_noalloc_streamed_landmark_chunks(esom):
    """Landmarks too large to stay resident in shared memory (d = 16,
    L = 2048: 136 KiB of rows) but within the scratch: the kernel streams
    them from the scratch in chunks and computes the pair distances from the
    rows.  Same coordinates as the handle path, and within the stated
    tolerance of the FP64 oracle, on two calls in a row."""
    import oracle
    from parity import coord_errors, report
    rng = np.random.default_rng(21)
    for seed in (0, 1):
        rng = np.random.default_rng(21 + seed)
        w = workloads.random_case(rng, 20_000, 16, 2048, 20, boost=1.5, adjust=1.0)
        X = torch.from_numpy(w.X).cuda()
        hi = torch.from_numpy(w.hi).cuda()
        lo = torch.from_numpy(w.lo).cuda()
        got = _noalloc(esom, w, X, hi, lo)
        with esom.Projector(w.d, w.L, w.k) as P:
            P.set_landmarks(hi, lo)
            assert P.config()["landmark_chunks"] > 1
            ref = P.project(X, w.boost, w.adjust)
            torch.cuda.synchronize()
        got, ref = got.cpu().numpy(), ref.cpu().numpy()
        err = np.abs(got.astype(np.float64) - ref).max()
        assert err <= COORD_TOL * w.extent, f"call {seed}: {err:.3e}"
        rows = np.arange(0, w.n, 10)
        o, ratio, _ = oracle.project(w.X[rows], w.hi, w.lo, w.k, w.boost, w.adjust,
                                     diagnostics=True)
        report(coord_errors(got[rows], o, ratio, w.extent), f"noalloc streamed, call {seed}")


def test_noalloc_takes_no_device_memory(esom):
    """After a first call (which looks up the scratch array's address), a call
    leaves the device's free memory unchanged: it allocates nothing."""
    w = workloads.mixture30_d16(seed=2, n=50_000)
    X = torch.from_numpy(w.X).cuda()
    hi = torch.from_numpy(w.hi).cuda()
    lo = torch.from_numpy(w.lo).cuda()
    out = torch.empty((w.n, 2), device="cuda")
    stream = torch.cuda.current_stream().cuda_stream

    def call():
        st = esom.esom_project_noalloc(X.data_ptr(), w.n, hi.data_ptr(), lo.data_ptr(), w.d,
                                       w.L, w.k, out.data_ptr(), w.boost, w.adjust, stream)
        assert st == esom.ESOM_OK, esom.esom_last_error()

    call()
    torch.cuda.synchronize()
    free0, _ = torch.cuda.mem_get_info()
    for _ in range(3):
        call()
    torch.cuda.synchronize()
    free1, _ = torch.cuda.mem_get_info()
    assert free1 == free0, f"free device memory changed by {free0 - free1} bytes"


def test_noalloc_rejects_landmarks_beyond_scratch(esom):
    d, L, k = 64, 20_000, 10          # 20000 * 66 * 4 bytes > 4 MiB of scratch
    X = torch.zeros((256, d), device="cuda")
    hi = torch.zeros((L, d), device="cuda")
    lo = torch.zeros((L, 2), device="cuda")
    out = torch.full((256, 2), 7.0, device="cuda")
    st = esom.esom_project_noalloc(X.data_ptr(), 256, hi.data_ptr(), lo.data_ptr(), d, L, k,
                                   out.data_ptr(), 1.0, 1.0, 0)
    assert st == esom.ESOM_EINVAL
    assert "scratch" in esom.esom_last_error()
    # k above the largest list a kernel is built for: the code esom_create gives
    st = esom.esom_project_noalloc(X.data_ptr(), 256, hi.data_ptr(), lo.data_ptr(), d, 100, 33,
                                   out.data_ptr(), 1.0, 1.0, 0)
    assert st == esom.ESOM_EUNSUPPORTED
    torch.cuda.synchronize()
    assert (out == 7.0).all()         # nothing was queued
