"""SOM landmark update and the frame server (GPU).

* esom_som_update against the FP64 oracle's batch SOM step on the same
  best-matching landmarks, its limits and its argument checks;
* the server's admission by device-memory budget;
* a served frame equal (bitwise) to the same steps issued by hand, and those
  steps against the oracle;
* a session's results equal (bitwise) alone and in a mix of sessions that
  run concurrently, frames of each session in order."""
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


def _stream():
    return torch.cuda.current_stream().cuda_stream


def _grid_case(d, side, b, seed):
    r = np.random.default_rng(seed)
    L = side * side
    hi = r.standard_normal((L, d)).astype(np.float32)
    lo = np.stack(np.meshgrid(np.arange(side), np.arange(side), indexing="ij"), -1)
    lo = lo.reshape(L, 2).astype(np.float32)
    batch = (r.standard_normal((b, d)) * 2).astype(np.float32)
    bmu = r.integers(0, L, b).astype(np.int32)
    return hi, lo, batch, bmu


def _som_gpu(esom, hi, lo, batch, bmu, alpha, sigma, stride=1):
    d, L = hi.shape[1], hi.shape[0]
    H = torch.from_numpy(hi).cuda()
    l = torch.from_numpy(lo).cuda()
    B = torch.from_numpy(batch).cuda()
    M = torch.from_numpy(np.ascontiguousarray(bmu)).cuda()
    b = batch.shape[0]
    st = esom.esom_som_update(H.data_ptr(), l.data_ptr(), d, L, B.data_ptr(), M.data_ptr(),
                              stride, b, alpha, sigma, _stream())
    assert st == 0, esom.esom_last_error()
    torch.cuda.synchronize()
    return H.cpu().numpy()


@pytest.mark.parametrize("d,side,sigma", [(8, 10, 1.5), (24, 16, 1.5), (24, 32, 3.0),
                                          (64, 8, 0.7), (4, 5, 1.0)])
def test_som_update_matches_oracle(esom, d, side, sigma):
    hi, lo, batch, bmu = _grid_case(d, side, 4096, 11 + d + side)
    for alpha in (0.05, 1.0):
        got = _som_gpu(esom, hi, lo, batch, bmu, alpha, sigma)
        want = oracle.som_step(hi, lo, batch, bmu, alpha, sigma)
        err = np.abs(got - want).max()
        scale = 1 + np.abs(batch).max()
        print(f"SOM d={d} L={side * side} sigma={sigma} alpha={alpha}: max err {err:.2e}")
        # FP32 weighted mean of 4096 points: a few ulps of the data scale
        assert err <= 2e-5 * scale


def test_som_update_bmu_from_knn(esom):
    """bmu taken with a stride from esom_knn's index output (column 0)."""
    w = workloads.serve_member(workloads.serve8(n_scale=0.05)[1])
    P = esom.Projector(w.d, w.L, w.k)
    hi, lo = torch.from_numpy(w.hi).cuda(), torch.from_numpy(w.lo).cuda()
    P.set_landmarks(hi, lo)
    X = torch.from_numpy(w.X[:4096].copy()).cuda()
    idx, _ = P.knn(X, with_dist=False)
    H = hi.clone()
    st = esom.esom_som_update(H.data_ptr(), lo.data_ptr(), w.d, w.L, X.data_ptr(),
                              idx.data_ptr(), w.k, X.shape[0], 0.05, 1.5, _stream())
    assert st == 0, esom.esom_last_error()
    torch.cuda.synchronize()
    bmu = idx[:, 0].cpu().numpy()
    oidx, od2 = oracle.knn(w.X[:4096], w.hi, 2)
    differ = np.nonzero(bmu != oidx[:, 0])[0]
    for i in differ:  # only ties of the nearest distance may differ
        dd = ((w.X[i].astype(np.float64) - w.hi[bmu[i]].astype(np.float64)) ** 2).sum()
        assert abs(dd - od2[i, 0]) <= 1e-6 * od2[i, 0]
    want = oracle.som_step(w.hi, w.lo, w.X[:4096], bmu, 0.05, 1.5)
    assert np.abs(H.cpu().numpy() - want).max() <= 2e-5 * (1 + np.abs(w.X[:4096]).max())


def test_som_update_limits_and_errors(esom):
    hi, lo, batch, bmu = _grid_case(16, 8, 1000, 5)
    bmu[::7] = 70  # beyond L: those points are skipped
    bmu[1::7] = -1
    keep = (bmu >= 0) & (bmu < 64)
    # b = 0 and alpha = 0 change nothing
    assert np.array_equal(_som_gpu(esom, hi, lo, batch[:0].copy(), bmu[:0].copy(), 0.5, 1.0), hi)
    assert np.array_equal(_som_gpu(esom, hi, lo, batch, bmu, 0.0, 1.0), hi)
    # sigma -> 0 in FP32 (neighbour weights underflow to 0): a k-means step
    got = _som_gpu(esom, hi, lo, batch, bmu, 1.0, 1e-3)
    for j in range(64):
        sel = keep & (bmu == j)
        if sel.any():
            mean = batch[sel].astype(np.float64).mean(0)
            assert np.abs(got[j] - mean).max() <= 1e-5 * (1 + np.abs(mean).max())
        else:
            assert np.array_equal(got[j], hi[j])
    # skipped entries count for nothing: same as dropping them
    ref = _som_gpu(esom, hi, lo, np.ascontiguousarray(batch[keep]), bmu[keep].copy(), 0.3, 1.0)
    want = oracle.som_step(hi, lo, batch[keep], bmu[keep], 0.3, 1.0)
    assert np.abs(ref - want).max() <= 2e-5 * (1 + np.abs(batch).max())
    # argument checks
    H = torch.from_numpy(hi).cuda()
    l = torch.from_numpy(lo).cuda()
    B = torch.from_numpy(batch).cuda()
    M = torch.from_numpy(bmu).cuda()
    args = dict(d=16, L=64, b=1000, alpha=0.5, sigma=1.0, stride=1)

    def call(**kw):
        a = dict(args, **kw)
        return esom.esom_som_update(H.data_ptr(), l.data_ptr(), a["d"], a["L"],
                                    kw.get("batch", B.data_ptr()), M.data_ptr(), a["stride"],
                                    a["b"], a["alpha"], a["sigma"], _stream())
    assert call(sigma=0.0) == esom.ESOM_EINVAL
    assert call(alpha=-1.0) == esom.ESOM_EINVAL
    assert call(d=6) == esom.ESOM_EINVAL
    assert call(stride=0) == esom.ESOM_EINVAL
    assert call(batch=B.data_ptr() + 4) == esom.ESOM_EALIGN
    torch.cuda.synchronize()
    assert np.array_equal(H.cpu().numpy(), hi)


def _session_arrays(p):
    w = workloads.serve_member(p)
    return w, torch.from_numpy(w.X), torch.from_numpy(w.hi), torch.from_numpy(w.lo)


def test_server_admission_by_budget(esom):
    ps = workloads.serve8(n_scale=0.02)
    w0, X0, h0, l0 = _session_arrays(ps[0])
    w1, X1, h1, l1 = _session_arrays(ps[1])
    with esom.Server(32 << 20, 2) as srv:
        a = srv.add_session(X0, h0, l0, w0.k, alpha=0.05, sigma=1.5, minibatch=4096)
        used, budget = srv.memory()
        assert 0 < used <= budget
        big = torch.from_numpy(np.tile(w1.X, (60, 1)))  # about 23 MB of points
        with pytest.raises(esom.EsomError) as e:
            srv.add_session(big, h1, l1, w1.k)
        assert e.value.status == esom.ESOM_ENOMEM
        assert "budget" in esom.esom_last_error()
        assert srv.memory()[0] == used
        b = srv.add_session(X1, h1, l1, w1.k)
        assert (a, b) == (0, 1)
        assert srv.memory()[0] > used
        with pytest.raises(esom.EsomError) as e:
            srv.add_session(X1, h1, l1, w1.k, boost=0.0)
        assert e.value.status == esom.ESOM_EINVAL
        srv.submit(a)
        srv.submit(b)
        recs = srv.poll(wait_all=True)
        assert sorted(r[0] for r in recs) == [0, 1]


def _manual_frames(esom, w, frames, alpha, sigma):
    """The server's frame steps issued by hand (minibatch = n, so the window
    is the whole point set every frame)."""
    P = esom.Projector(w.d, w.L, w.k)
    hi, lo = torch.from_numpy(w.hi).cuda(), torch.from_numpy(w.lo).cuda()
    P.set_landmarks(hi, lo)
    X = torch.from_numpy(w.X).cuda()
    out = None
    his = []
    for _ in range(frames):
        idx, _ = P.knn(X, with_dist=False)
        st = esom.esom_som_update(hi.data_ptr(), lo.data_ptr(), w.d, w.L, X.data_ptr(),
                                  idx.data_ptr(), w.k, w.n, alpha, sigma, _stream())
        assert st == 0, esom.esom_last_error()
        P.set_landmarks(hi, lo)
        out = P.project(X, w.boost, w.adjust)
        his.append((hi.cpu().numpy().copy(), idx[:, 0].cpu().numpy()))
    torch.cuda.synchronize()
    P.close()
    return out, his


def test_served_frames_equal_manual_steps_and_oracle(esom):
    p = dict(workloads.serve8(n_scale=0.01)[3])  # L=1024, n=10,000
    w, X, h, l = _session_arrays(p)
    frames, alpha, sigma = 3, 0.05, 1.5
    with esom.Server(1 << 30, 1) as srv:
        s = srv.add_session(X, h, l, w.k, w.boost, w.adjust, alpha, sigma, minibatch=w.n)
        for _ in range(frames):
            srv.submit(s)
        recs = srv.poll(wait_all=True)
        assert [r[1] for r in recs] == list(range(frames))
        got, done = srv.output(s)
        assert done == frames
    want, his = _manual_frames(esom, w, frames, alpha, sigma)
    assert torch.equal(got, want)
    # the first SOM step against the oracle's, on the same best matches
    hi1, bmu0 = his[0]
    ref = oracle.som_step(w.hi, w.lo, w.X, bmu0, alpha, sigma)
    assert np.abs(hi1 - ref).max() <= 2e-5 * (1 + np.abs(w.X).max())
    # the last frame's projection against the oracle on the device's landmarks
    hiN = his[-1][0]
    ref, ratio, _ = oracle.project(w.X, hiN, w.lo, w.k, w.boost, w.adjust, diagnostics=True)
    stats = coord_errors(got.cpu().numpy(), ref, ratio, w.extent)
    report(stats, f"served frame {frames}")


def test_served_trajectory_against_oracle_only(esom):
    """Three served frames against a trajectory computed by the oracle alone
    (its exact best-matching landmarks, its FP64 SOM step, its projection of
    the final landmarks), with nothing taken from the GPU: the coordinates
    after the last frame agree within the projection's parity bar."""
    p = dict(workloads.serve8(n_scale=0.01)[2])  # L=256, n=2,000
    w, X, h, l = _session_arrays(p)
    frames, alpha, sigma = 3, 0.05, 1.5
    with esom.Server(1 << 30, 1) as srv:
        s = srv.add_session(X, h, l, w.k, w.boost, w.adjust, alpha, sigma, minibatch=w.n)
        for _ in range(frames):
            srv.submit(s)
        srv.poll(wait_all=True)
        got, done = srv.output(s)
        assert done == frames
    hi = w.hi.astype(np.float64)
    for _ in range(frames):
        idx, _ = oracle.knn(w.X, hi.astype(np.float32), 2)  # the oracle's k-NN wants k >= 2
        hi = oracle.som_step(hi, w.lo, w.X, idx[:, 0].astype(np.int32), alpha, sigma)
    ref, ratio, _ = oracle.project(w.X, hi.astype(np.float32), w.lo, w.k, w.boost, w.adjust,
                                   diagnostics=True)
    stats = coord_errors(got.cpu().numpy(), ref, ratio, w.extent)
    report(stats, f"served {frames} frames vs the oracle's own trajectory")


def test_session_alone_equals_in_mix(esom):
    """Session 0's outputs after four frames (SOM window from the seed and the
    frame number) are bitwise the same served alone and served concurrently
    with three other sessions; every session's frames complete in order."""
    ps = workloads.serve8(n_scale=0.02)[:4]
    arrs = [_session_arrays(p) for p in ps]
    frames = 4

    def add(srv, i):
        w, X, h, l = arrs[i]
        p = ps[i]
        Xd = X.cuda() if i % 2 else X  # device and host sources both work
        return srv.add_session(Xd, h, l, w.k, w.boost, w.adjust, p["alpha"], p["sigma"],
                               minibatch=p["minibatch"], seed=p["seed"])

    with esom.Server(1 << 30, 1) as srv:
        s = add(srv, 0)
        for _ in range(frames):
            srv.submit(s)
        srv.poll(wait_all=True)
        alone, _ = srv.output(s)
    with esom.Server(1 << 30, 4) as srv:
        sids = [add(srv, i) for i in range(4)]
        t = srv.now()
        for f in range(frames):
            for i in reversed(sids):
                srv.submit(i, t + 0.001 * (4 * f + i))
        recs = srv.poll(wait_all=True)
        mixed = [srv.output(i) for i in sids]
    assert torch.equal(mixed[0][0], alone)
    assert all(m[1] == frames for m in mixed)
    for i in sids:
        own = [r for r in recs if r[0] == i]
        assert [r[1] for r in own] == list(range(frames))
        comp = [r[3] for r in own]
        assert comp == sorted(comp)
    assert len(recs) == 4 * frames


def test_fifo_start_order(esom):
    """With one slot, queued frames start by arrival time, not submission."""
    ps = workloads.serve8(n_scale=0.005)[:3]
    arrs = [_session_arrays(p) for p in ps]
    with esom.Server(1 << 30, 1) as srv:
        sids = [srv.add_session(X, h, l, w.k) for (w, X, h, l) in arrs]
        srv.submit(sids[0], 10.0)  # starts at once: the slot is free
        srv.submit(sids[1], 12.0)
        srv.submit(sids[2], 11.0)
        recs = srv.poll(wait_all=True)
    order = [r[0] for r in sorted(recs, key=lambda r: r[3])]
    assert order == [sids[0], sids[2], sids[1]]


def test_coalesced_frames_equal_strict(esom):
    """Coalescing runs queued frames' SOM steps in order and projects once:
    the final output equals frame-by-frame serving bit for bit, and every
    frame is reported, in order."""
    ps = workloads.serve8(n_scale=0.02)[:2]
    arrs = [_session_arrays(p) for p in ps]
    frames = 6
    outs = []
    for coalesce in (False, True):
        with esom.Server(1 << 30, 1) as srv:
            srv.set_coalescing(coalesce)
            sids = []
            for (w, X, h, l), p in zip(arrs, ps):
                sids.append(srv.add_session(X, h, l, w.k, w.boost, w.adjust, p["alpha"],
                                            p["sigma"], minibatch=p["minibatch"], seed=p["seed"]))
            for f in range(frames):
                for s in sids:
                    srv.submit(s)
            recs = srv.poll(wait_all=True)
            outs.append([srv.output(s) for s in sids])
            for s in sids:
                own = [r for r in recs if r[0] == s]
                assert [r[1] for r in own] == list(range(frames))
            if coalesce:
                # frames queued behind the first were started together
                comp = sorted({round(r[3], 9) for r in recs if r[0] == sids[0]})
                assert len(comp) < frames
    for (a, fa), (b, fb) in zip(outs[0], outs[1]):
        assert fa == fb == frames
        assert torch.equal(a, b)


def test_server_tf32_sessions_equal_fp32(esom):
    """Sessions whose handles screen on the tensor cores give the same bits."""
    p = workloads.serve8(n_scale=0.01)[3]
    w, X, h, l = _session_arrays(p)
    outs = []
    for mode in (esom.ESOM_SCREEN_FP32, esom.ESOM_SCREEN_TF32):
        with esom.Server(1 << 30, 2) as srv:
            srv.set_screening(mode)
            s = srv.add_session(X, h, l, w.k, w.boost, w.adjust, p["alpha"], p["sigma"],
                                minibatch=p["minibatch"], seed=p["seed"])
            for _ in range(3):
                srv.submit(s)
            srv.poll(wait_all=True)
            outs.append(srv.output(s)[0])
            with pytest.raises(esom.EsomError):
                srv.set_screening(esom.ESOM_SCREEN_FP32)  # sessions exist already
    assert torch.equal(outs[0], outs[1])


def test_server_auto_screening_equals_fp32(esom):
    """Sessions tuned automatically at admission give the FP32 sessions' bits."""
    ps = workloads.serve8(n_scale=0.01)[:2]
    outs = []
    for mode in (esom.ESOM_SCREEN_FP32, esom.ESOM_SCREEN_AUTO):
        with esom.Server(1 << 30, 2) as srv:
            srv.set_screening(mode)
            sids = []
            for p in ps:
                w, X, h, l = _session_arrays(p)
                sids.append(srv.add_session(X, h, l, w.k, w.boost, w.adjust, p["alpha"],
                                            p["sigma"], minibatch=p["minibatch"], seed=p["seed"]))
            for _ in range(2):
                for s in sids:
                    srv.submit(s)
            srv.poll(wait_all=True)
            outs.append([srv.output(s)[0] for s in sids])
    for a, b in zip(outs[0], outs[1]):
        assert torch.equal(a, b)
