"""The paper's alternative kernel designs (GPU): the Base and Bitonic k-NN
kernels (Section 4.2) return esom_knn's neighbours and distances bit for
bit; the library's projection kernel run on esom_knn's neighbours returns
esom_project's bits; the Registers projection (Section 4.3: a warp per
point, pairs in 2 x 2 blocks, D_uv by direct dot products) agrees with the
FP64 oracle within twice the library's coordinate tolerance.  (Its D_uv =
<X - L_u, L_v - L_u> / |L_v - L_u|^2 is an FP32 dot product over d terms,
where the library's law-of-cosines form starts from the exact squared
distances; on nearly singular systems the difference is amplified.)"""
import json

import numpy as np
import pytest

import oracle
from parity import COORD_TOL, coord_errors, report
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


def case(name):
    r = np.random.default_rng(sum(map(ord, name)))
    if name == "mixture10_d8":
        return workloads.mixture10_d8()
    if name == "mixture30_d16":
        return workloads.mixture30_d16(n=20_077)
    if name == "student50_d32":
        return workloads.make("student50_d32", n=3000)
    if name == "d64_k20":
        return workloads.random_case(r, 3000, 64, 333, 20, boost=1.5, adjust=0.5)
    if name == "d4_k2":
        return workloads.random_case(r, 2000, 4, 300, 2)
    if name == "d12_k32":
        return workloads.random_case(r, 2000, 12, 70, 32)
    if name == "L_equals_k":
        return workloads.random_case(r, 1000, 32, 5, 5)
    if name == "n1":
        w = workloads.random_case(r, 1, 16, 100, 7)
        return w
    if name == "n33_k3":
        return workloads.random_case(r, 33, 20, 64, 3)
    raise KeyError(name)


CASES = ["mixture10_d8", "mixture30_d16", "student50_d32", "d64_k20", "d4_k2", "d12_k32",
         "L_equals_k", "n1", "n33_k3"]


def check_registers(w, out, label):
    ref, ratio, _ = oracle.project(w.X, w.hi, w.lo, w.k, w.boost, w.adjust, diagnostics=True)
    stats = coord_errors(out, ref, ratio, w.extent, tol=2 * COORD_TOL)
    report(stats, label)


def projector(esom, w, centering=False):
    P = esom.Projector(w.d, w.L, w.k)
    P.set_centering(centering)
    P.set_landmarks(torch.from_numpy(w.hi).cuda(), torch.from_numpy(w.lo).cuda())
    return P


@pytest.mark.parametrize("name", CASES)
def test_knn_variants_equal_library(esom, name):
    w = case(name)
    X = torch.from_numpy(w.X).cuda()
    with projector(esom, w) as P:
        idx, d2 = P.knn(X)
        got = {v: P.knn_variant(X, v) for v in (esom.ESOM_KNN_BASE, esom.ESOM_KNN_BITONIC)}
        torch.cuda.synchronize()
        assert P.device_status() == 0
    for v, (gi, gd) in got.items():
        assert torch.equal(gi, idx), f"variant {v}: indices differ"
        assert torch.equal(gd.view(torch.int32), d2.view(torch.int32)), f"variant {v}: distances"


@pytest.mark.parametrize("name", CASES)
def test_projection_variants(esom, name):
    w = case(name)
    X = torch.from_numpy(w.X).cuda()
    with projector(esom, w) as P:
        ref = P.project(X, w.boost, w.adjust)
        idx, d2 = P.knn(X)
        table = P.project_knn(X, idx, d2, esom.ESOM_PROJ_TABLE, w.boost, w.adjust)
        regs = P.project_knn(X, idx, d2, esom.ESOM_PROJ_REGISTERS, w.boost, w.adjust)
        torch.cuda.synchronize()
        assert P.device_status() == 0
    assert torch.equal(table.view(torch.int32), ref.view(torch.int32))
    if w.k >= 3:  # k = 2 has one scored neighbour and no pairs
        check_registers(w, regs.cpu().numpy(), f"registers {name}")
    else:
        assert torch.equal(regs, ref)


def test_variants_with_centring(esom):
    """Centred handles: the variants load points through the same centre."""
    w = workloads.random_case(np.random.default_rng(8), 3000, 16, 256, 12)
    w.X = (w.X + 300.0).astype(np.float32)
    w.hi = (w.hi + 300.0).astype(np.float32)
    X = torch.from_numpy(w.X).cuda()
    with projector(esom, w, centering=True) as P:
        idx, d2 = P.knn(X)
        bi, bd = P.knn_variant(X, esom.ESOM_KNN_BITONIC)
        ref = P.project(X, w.boost, w.adjust)
        regs = P.project_knn(X, idx, d2, esom.ESOM_PROJ_REGISTERS, w.boost, w.adjust)
        torch.cuda.synchronize()
    assert torch.equal(bi, idx) and torch.equal(bd, d2)
    check_registers(w, regs.cpu().numpy(), "registers centred")
    assert ref.shape == regs.shape


def test_variant_errors(esom):
    w = case("d4_k2")
    X = torch.from_numpy(w.X).cuda()
    with projector(esom, w) as P:
        idx, d2 = P.knn(X)
        with pytest.raises(esom.EsomError) as e:
            P.knn_variant(X, 7)
        assert e.value.status == esom.ESOM_EINVAL
        with pytest.raises(esom.EsomError) as e:
            P.project_knn(X, idx, d2, 5)
        assert e.value.status == esom.ESOM_EINVAL
        # neighbour rows 4 bytes off a 16-byte boundary
        flat_i = torch.zeros(X.shape[0] * w.k + 1, dtype=torch.int32, device="cuda")
        off_i = flat_i[1:].view(X.shape[0], w.k)
        off_i.copy_(idx)
        with pytest.raises(esom.EsomError) as e:
            P.project_knn(X, off_i, d2)
        assert e.value.status == esom.ESOM_EALIGN
        # zero points: no launch
        empty = X[:0]
        P.knn_variant(empty, esom.ESOM_KNN_BASE)
        P.project_knn(empty, idx[:0], d2[:0])
        torch.cuda.synchronize()
        assert P.device_status() == 0
