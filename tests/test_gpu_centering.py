"""Opt-in centring (esom_set_centering) on data far from the origin (GPU).

The screening certificate's error bound grows with |x| max|l|, so shifted
data fail it and are rescanned exactly.  Centred on the landmarks' rounded
mean, the same data screen as well as unshifted data; distances are
unchanged up to FP32 rounding, so results stay within the oracle's
tolerance, and every execution plan still gives the same bits."""
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


def shifted(shift=200.0, n=6000, d=16, L=512, k=12, seed=11):
    w = workloads.random_case(np.random.default_rng(seed), n, d, L, k)
    w.X = (w.X + shift).astype(np.float32)
    w.hi = (w.hi + shift).astype(np.float32)
    return w


def run(esom, w, centering, plan, chunk=None):
    X = torch.from_numpy(w.X).cuda()
    with esom.Projector(w.d, w.L, w.k) as P:
        P.set_centering(centering)
        P.set_landmarks(torch.from_numpy(w.hi).cuda(), torch.from_numpy(w.lo).cuda())
        if chunk:
            P.set_landmark_chunk(chunk)
        P.set_plan(plan)
        out = P.project(X, w.boost, w.adjust).cpu().numpy()
        idx, d2 = P.knn(X)
        torch.cuda.synchronize()
        assert P.device_status() == 0
        cfg = P.config()
        cfg["stats"] = P.stats()
    return out, idx.cpu().numpy(), d2.cpu().numpy(), cfg


def frac(cfg):
    return cfg["stats"]["rescans"] / max(cfg["stats"]["points"], 1)


@pytest.mark.parametrize("mode", ["tf32", "bf16"])
def test_centring_removes_rescans(esom, mode):
    plan = {"tf32": esom.ESOM_PLAN_TF32, "bf16": esom.ESOM_PLAN_BF16}[mode]
    w = shifted()
    plain = run(esom, w, False, plan)
    cent = run(esom, w, True, plan)
    print("CENTRING", mode, "rescans plain", frac(plain[3]), "centred", frac(cent[3]))
    assert frac(plain[3]) > 0.5
    assert frac(cent[3]) <= 0.2
    check(w, *cent[:3], label=f"centred {mode}", named=False)


@pytest.mark.parametrize("chunk", [None, 200])
def test_centred_plans_agree_and_match_oracle(esom, chunk):
    """Fused, split, TF32 and BF16 with centring: one set of bits, within
    the oracle's tolerance; also with the landmarks streamed in chunks."""
    w = shifted(shift=-350.0, seed=5)
    outs = {}
    for plan in esom.PLAN_NAMES:
        out, idx, d2, cfg = run(esom, w, True, plan, chunk=chunk)
        outs[plan] = out
        if plan == esom.ESOM_PLAN_FUSED:
            check(w, out, idx, d2, label=f"centred fused chunk={chunk}", named=False)
    ref = outs[esom.ESOM_PLAN_FUSED]
    for o in outs.values():
        assert np.array_equal(o.view(np.uint32), ref.view(np.uint32))


def test_centring_keeps_integer_data_exact(esom):
    """Integer coordinates stay integers after subtracting an integer
    centre, so the squared distances, and with them the neighbours, are
    the exact ones."""
    r = np.random.default_rng(3)
    w = workloads.random_case(r, 3000, 8, 200, 10)
    w.X = (np.round(w.X * 50.0) + 1000.0).astype(np.float32)
    w.hi = (np.round(w.hi * 50.0) + 1000.0).astype(np.float32)
    out, idx, d2, cfg = run(esom, w, True, esom.ESOM_PLAN_TF32)
    Xd = w.X.astype(np.float64)
    Hd = w.hi.astype(np.float64)
    got = ((Xd[:, None, :] - Hd[idx]) ** 2).sum(-1)
    assert np.array_equal(got, d2.astype(np.float64))
    full = ((Xd[:, None, :] - Hd[None, :, :]) ** 2).sum(-1)
    kth = np.sort(full, axis=1)[:, w.k - 1]
    assert (got.max(axis=1) == kth).all()


def test_setting_takes_effect_at_set_landmarks(esom):
    """Turning centring on after the landmarks are stored changes nothing
    until they are stored again."""
    w = shifted(n=2000)
    X = torch.from_numpy(w.X).cuda()
    hi = torch.from_numpy(w.hi).cuda()
    lo = torch.from_numpy(w.lo).cuda()
    with esom.Projector(w.d, w.L, w.k) as P:
        P.set_landmarks(hi, lo)
        a = P.project(X, w.boost, w.adjust).clone()
        P.set_centering(True)
        b = P.project(X, w.boost, w.adjust).clone()
        P.set_landmarks(hi, lo)
        c = P.project(X, w.boost, w.adjust).clone()
        P.set_centering(False)
        P.set_landmarks(hi, lo)
        d = P.project(X, w.boost, w.adjust).clone()
        torch.cuda.synchronize()
        assert P.device_status() == 0
    assert torch.equal(a, b) and torch.equal(a, d)
    # centred results differ only by rounding
    assert torch.allclose(a, c, atol=1e-3 * w.extent, rtol=0)
