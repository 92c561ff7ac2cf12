"""The bounded device waits and the FP64 reciprocal of the solve (GPU).

A wait that runs out must leave a status the host can read and a usable
context: esom_test_stall arms one launch of the fused kernel to wait on a
barrier that nothing completes (bounded, 1 ms), so the kernel takes its
timeout path for real, without any fault.  The reciprocal (an SFU estimate
refined by two Newton steps, used by Cramer's rule, Section 3.1 step 4) is
compared with CUDA's own division over the determinants the solve meets."""
import numpy as np
import pytest

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


def test_wait_that_runs_out_reports_edevice(esom):
    w = workloads.mixture10_d8(n=5000)
    with esom.Projector(w.d, w.L, w.k) as P:
        P.set_landmarks(torch.from_numpy(w.hi).cuda(), torch.from_numpy(w.lo).cuda())
        P.set_plan(esom.ESOM_PLAN_FUSED)
        X = torch.from_numpy(w.X).cuda()
        ref = P.project(X, w.boost, w.adjust)
        torch.cuda.synchronize()
        assert esom.esom_device_status(P.h, 0) == esom.ESOM_OK
        # the probe needs the fused plan
        P.set_plan(esom.ESOM_PLAN_SPLIT)
        assert esom.esom_test_stall(P.h, 1_000_000) == esom.ESOM_EINVAL
        P.set_plan(esom.ESOM_PLAN_FUSED)
        assert esom.esom_test_stall(P.h, 10) == esom.ESOM_EINVAL
        assert esom.esom_test_stall(P.h, 1_000_000) == esom.ESOM_OK
        out = torch.full_like(ref, 12345.0)
        P.project(X, w.boost, w.adjust, out=out)
        torch.cuda.synchronize()
        assert esom.esom_device_status(P.h, 0) == esom.ESOM_EDEVICE
        assert "bounded wait" in esom.esom_last_error()
        # no block wrote its points
        assert (out == 12345.0).all()
        # the status is cleared by the read, the context and the handle
        # stay usable, and the probe was consumed by the one launch
        assert esom.esom_device_status(P.h, 0) == esom.ESOM_OK
        again = P.project(X, w.boost, w.adjust)
        torch.cuda.synchronize()
        assert esom.esom_device_status(P.h, 0) == esom.ESOM_OK
        assert torch.equal(again, ref)


def test_drcp_against_cuda_division(esom):
    """Relative difference of the solve's reciprocal from CUDA's correctly
    rounded 1.0 / x, in units of the last place, over log-uniform |x| in
    [1e-80, 1e80] (FP32 normal-matrix entries give determinants well inside
    that range), powers of two and values next to them."""
    rng = np.random.default_rng(5)
    x = 10.0 ** rng.uniform(-80, 80, 200_000)
    x *= rng.choice([-1.0, 1.0], x.size)
    p2 = 2.0 ** np.arange(-260, 261, dtype=np.float64)
    x = np.concatenate([x, p2, np.nextafter(p2, 0), np.nextafter(p2, np.inf), -p2,
                        [1.0, 3.0, 7.0, 1.0 / 3.0, 0.1, 1e-300 * 1e220]])
    xd = torch.from_numpy(x).cuda()
    rcp, div = torch.empty_like(xd), torch.empty_like(xd)
    assert esom.esom_selftest_drcp(xd.data_ptr(), x.size, rcp.data_ptr(), div.data_ptr(),
                                   torch.cuda.current_stream().cuda_stream) == esom.ESOM_OK
    torch.cuda.synchronize()
    r, q = rcp.cpu().numpy(), div.cpu().numpy()
    assert np.array_equal(q, 1.0 / x)            # CUDA's division: correctly rounded
    ulp = np.abs(r - q) / np.spacing(np.abs(q))
    print(f"DRCP max ulp {ulp.max():.3f}, mean {ulp.mean():.3e}, "
          f"exact {np.mean(r == q):.4f} of {x.size}")
    assert ulp.max() <= 1.0
