"""The error model behind the tensor-core certificate, measured (GPU).

The screened k-NN ranks landmarks by v_j = |L_j|^2 - 2 T_j with T_j = x . L_j
accumulated by the tensor cores from split operands (x = x_hi + x_lo, TF32
or BF16 parts; Section 4.2's distance block as a tcgen05 contraction).  The
kernel's certificate assumes |2 T_j - 2 x . L_j| <= tc_dot_bound |x| max|l|
with tc_dot_bound = 4 (3 2^-2p + (3d + 1) 2^-23): the split's dropped terms
and 3d FP32 roundings relative to the sum of |products|, doubled for v and
doubled again as a margin.  Here the raw accumulator values are read back
(esom_selftest_tc_products) on rows whose coordinates span 2^-10 .. 2^10, and
on rows with one dominant coordinate, and the measured error must stay within
half of that bound: the model itself, without its margin, must hold."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def esom():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2201_00701_gb300 import binding
    binding.load(build_if_missing=True)
    return binding


def wide_rows(rng, n, d):
    """Half the rows: every coordinate 2^U[-10, 10] with a random sign; half:
    one coordinate of magnitude 2^10, the rest 2^U[-10, 0]."""
    mag = 2.0 ** rng.uniform(-10, 10, (n, d))
    dom = 2.0 ** rng.uniform(-10, 0, (n, d))
    dom[np.arange(n), rng.integers(0, d, n)] = 2.0 ** 10
    X = np.where((np.arange(n) % 2 == 0)[:, None], mag, dom)
    X *= rng.choice([-1.0, 1.0], (n, d))
    return X.astype(np.float32)


def tc_dot_bound(d, mode):
    split = 2.0 ** -16 if mode == "bf16" else 2.0 ** -22    # 2^-2p, p = 8 or 11
    return 4.0 * (3.0 * split + (3 * d + 1) * 2.0 ** -23)


@pytest.mark.parametrize("mode", ["tf32", "bf16"])
@pytest.mark.parametrize("d", [8, 16, 48])
def test_tensor_core_products_within_model(esom, d, mode):
    rng = np.random.default_rng(100 + d)
    n, L = 640, 200
    X = wide_rows(rng, n, d)
    hi = wide_rows(rng, L, d)
    lo = rng.uniform(0, 10, (L, 2)).astype(np.float32)
    with esom.Projector(d, L, 10) as P:
        P.set_landmarks(torch.from_numpy(hi).cuda(), torch.from_numpy(lo).cuda())
        P.set_screening({"tf32": esom.ESOM_SCREEN_TF32, "bf16": esom.ESOM_SCREEN_BF16}[mode])
        Lc = 64 * ((L + 63) // 64)
        T = torch.full((n, Lc), float("nan"), device="cuda")
        Xd = torch.from_numpy(X).cuda()
        st = esom.esom_selftest_tc_products(P.h, Xd.data_ptr(), n, T.data_ptr(),
                                            torch.cuda.current_stream().cuda_stream)
        assert st == esom.ESOM_OK, esom.esom_last_error()
        torch.cuda.synchronize()
        assert P.device_status() == 0
        T = T.cpu().numpy().astype(np.float64)
    exact = X.astype(np.float64) @ hi.astype(np.float64).T            # n x L, exact products
    assert np.all(T[:, L:] == 0.0)                                     # zero padding rows
    xn = np.linalg.norm(X.astype(np.float64), axis=1)
    lmax = np.linalg.norm(hi.astype(np.float64), axis=1).max()
    # error of v_j = |l|^2 - 2 T_j per unit |x| max|l|, against the bound
    ratio = 2.0 * np.abs(T[:, :L] - exact) / (xn[:, None] * lmax)
    bound = tc_dot_bound(d, mode)
    print(f"TCBOUND d={d} {mode}: max error {ratio.max():.3e} = "
          f"{ratio.max() / bound:.3f} of the certificate bound {bound:.3e}")
    assert ratio.max() <= 0.5 * bound
