"""The learned warm start and block LOBPCG (eigenvectors of eq. (Zi) for
partial selections) against the CPU oracles.

Bars:
  * features: the oracle's definitions in FP64, compared after the library's
    rounding to FP32 (relative 1e-5, absolute 1e-5);
  * target projectors B^T Q Q^T B: 1e-6 absolute (both sides build the same
    Krylov basis by classical Gram-Schmidt applied twice in FP64);
  * MLP forward and gradient against the FP64 oracle with the same
    bfloat16-rounded weights: 1e-4 relative (FP32 accumulation over at most
    256 terms per output, and over the batch for the gradient);
  * one Adam step: 1e-6 relative on the master weights, and the bfloat16
    copy equal to the oracle's rounding of the GPU master weights;
  * LOBPCG eigenvectors (plain FP64 form): every partial subdomain accepted,
    apply within 1e-8 of the oracle's (residual tolerance 1e-9 on T, whose
    wanted eigenvalues are separated from the rest by the threshold tau), PCG
    iterations +-1;
  * learned start: accepted results, the same preconditioner quality (PCG
    iterations +-1), the condition estimate under the Sec. 3.2 bound, and the
    measured LOBPCG iteration counts with and without the network reported.
"""
import numpy as np
import pytest

import synth
from oracle import amdd_oracle as O
from oracle import proposal as L

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

from paper_2109_05908_gb300 import amdd as A  # noqa: E402
from paper_2109_05908_gb300 import learned as Lg  # noqa: E402
from paper_2109_05908_gb300.device import DeviceMatrix, stream_ptr, to_device  # noqa: E402


def _diff(m, N, seed, ov, tau, lo, hi):
    M = synth.diffusion3d(m, sigma=1.0, corr=2.0, n_channels=2, seed=seed, channel_value=1e3)
    part = synth.bfs_partition(M, N, seed=seed, min_size=lo, max_size=hi)
    return M, part, int(part.max()) + 1, ov, tau


def _setup(prob, precision=0, eig_solver=0, keep=0, opts=None):
    M, part, N, ov, tau = prob
    dA = DeviceMatrix(M)
    dpart = torch.from_numpy(np.asarray(part, np.int32)).cuda()
    o = opts if opts is not None else A.opts_default()
    o.precision = precision
    if opts is None:
        o.eig_solver = eig_solver
    o.keep_proposal_data = keep
    h = A.setup(dA.csr, dpart.data_ptr(), N, ov, tau, o, stream_ptr())
    return h, (dA, dpart)


def test_features_and_targets_match_oracle():
    prob = _diff(8, 6, 1, 1, 0.5, 40, 160)
    M, part, N, ov, tau = prob
    h, keep = _setup(prob, keep=1)
    try:
        feat, tgt, sub = A.proposal_export(h)
    finally:
        A.destroy(h)
    S = O.setup(M, part, N, ov, tau)
    assert len(sub) == sum(1 for s in S.subs if 0 < s.p < len(s.I)) and len(sub) > 0
    for q, i in enumerate(sub):
        s = S.subs[i]
        fo = L.features(s.Aii, len(s.I), len(s.G), len(s.D), s.p, tau)
        assert np.allclose(feat[q], fo, rtol=1e-5, atol=1e-5), (i, np.abs(feat[q] - fo).max())
        B = L.krylov_basis(s.Aii[: len(s.I), : len(s.I)])
        to = L.target_projector(B, s.Z[: len(s.I)])
        assert np.abs(tgt[q] - to).max() <= 1e-6


def _bf16_params(seed=0):
    w = Lg.init_weights(seed).astype(np.float64) * 0.7
    return L.bf16(w).astype(np.float32)


def _oracle_params(wb):
    o = {}
    off = 0
    for name, shape in (("W1", (32, 256)), ("b1", (256,)), ("W2", (256, 256)), ("b2", (256,)), ("W3", (256, 256)),
                        ("b3", (256,))):
        size = int(np.prod(shape))
        o[name] = wb[off: off + size].astype(np.float64).reshape(shape)
        off += size
    return o


def test_mlp_forward_and_gradient_match_oracle():
    rng = np.random.default_rng(5)
    n = 24
    wb = _bf16_params(1)
    wb[L.NF * 256: L.NF * 256 + 256] = rng.standard_normal(256).astype(np.float32) * 0.05  # non-zero biases
    wb = L.bf16(wb).astype(np.float32)
    X = rng.standard_normal((n, 32)).astype(np.float32)
    Qt = rng.standard_normal((n, 16, 16)).astype(np.float32)
    Qt = 0.5 * (Qt + Qt.transpose(0, 2, 1))
    P = _oracle_params(wb)
    Qo, cache = L.forward(P, X.astype(np.float64))
    go = L.backward(P, Qo, Qt.astype(np.float64), cache)
    dwb, dX, dQt = to_device(wb), to_device(X), to_device(Qt.reshape(n, -1))
    _, nwork = A.mlp_sizes(n)
    work = torch.empty(nwork, dtype=torch.float32, device="cuda")
    q = torch.empty((n, 256), dtype=torch.float32, device="cuda")
    A.mlp_forward(dwb.data_ptr(), dX.data_ptr(), n, q.data_ptr(), work.data_ptr(), stream_ptr())
    qg = q.cpu().numpy().reshape(n, 16, 16)
    assert np.abs(qg - Qo).max() <= 1e-4 * max(1.0, np.abs(Qo).max())
    grad = torch.empty(A.MLP_NPARAM, dtype=torch.float32, device="cuda")
    loss = torch.empty(1, dtype=torch.float32, device="cuda")
    A.mlp_train_step(0, dwb.data_ptr(), 0, 0, 0, 0.0, dX.data_ptr(), dQt.data_ptr(), n, grad.data_ptr(),
                     work.data_ptr(), loss.data_ptr(), stream_ptr())
    assert abs(float(loss.item()) - L.loss(Qo, Qt.astype(np.float64))) <= 1e-4 * L.loss(Qo, Qt.astype(np.float64))
    gg = grad.cpu().numpy()
    ref = np.concatenate([go[k].reshape(-1) for k in ("W1", "b1", "W2", "b2", "W3", "b3")])
    assert np.abs(gg - ref).max() <= 1e-4 * max(1.0, np.abs(ref).max())


def test_adam_step_matches_oracle():
    rng = np.random.default_rng(6)
    n = 16
    w = Lg.init_weights(2)
    wb = L.bf16(w).astype(np.float32)
    X = rng.standard_normal((n, 32)).astype(np.float32)
    Qt = rng.standard_normal((n, 16, 16)).astype(np.float32)
    Qt = 0.5 * (Qt + Qt.transpose(0, 2, 1))
    dw, dwb = to_device(w), to_device(wb)
    dm = torch.zeros_like(dw)
    dv = torch.zeros_like(dw)
    dX, dQt = to_device(X), to_device(Qt.reshape(n, -1))
    _, nwork = A.mlp_sizes(n)
    work = torch.empty(nwork, dtype=torch.float32, device="cuda")
    grad = torch.empty(A.MLP_NPARAM, dtype=torch.float32, device="cuda")
    loss = torch.empty(1, dtype=torch.float32, device="cuda")
    lr = 1e-3
    A.mlp_train_step(dw.data_ptr(), dwb.data_ptr(), dm.data_ptr(), dv.data_ptr(), 1, lr, dX.data_ptr(),
                     dQt.data_ptr(), n, grad.data_ptr(), work.data_ptr(), loss.data_ptr(), stream_ptr())
    g = grad.cpu().numpy().astype(np.float64)
    Po = {"w": w.astype(np.float64)}
    L.adam_step(Po, {"w": g}, {}, lr)
    wn = dw.cpu().numpy()
    assert np.allclose(wn, Po["w"], rtol=1e-6, atol=1e-7)
    assert np.array_equal(dwb.cpu().numpy(), L.bf16(wn).astype(np.float32))


def _apply_err(h, S, M):
    r = synth.rhs(M.n, 9)
    zo = O.apply(S, r)
    rd = to_device(r)
    zd = torch.empty_like(rd)
    A.apply(h, rd.data_ptr(), zd.data_ptr(), 1)
    return np.linalg.norm(zd.cpu().numpy() - zo) / np.linalg.norm(zo)


def _pcg_its(h, M):
    bd = to_device(synth.rhs(M.n, 0))
    x = torch.zeros_like(bd)
    return A.pcg_solve(h, bd.data_ptr(), x.data_ptr(), 1, 1e-8, 1000)


@pytest.mark.parametrize("precision,bar", [(0, 1e-8), (2, 1e-3)])
def test_lobpcg_cold_start_matches_oracle(precision, bar):
    prob = _diff(8, 6, 1, 1, 0.5, 40, 160)
    M, part, N, ov, tau = prob
    S = O.setup(M, part, N, ov, tau)
    h, keep = _setup(prob, precision=precision, eig_solver=1)
    try:
        info = A.get_info(h)
        assert info.n_partial > 0 and info.lobpcg_subdomains == info.n_partial and info.lobpcg_fallbacks == 0
        its = A.eig_iterations(h, N)
        assert np.all(its[[i for i, s in enumerate(S.subs) if 0 < s.p < len(s.I)]] >= 0)
        for i, s in enumerate(S.subs):
            assert A.get_subdomain(h, i)[3] == s.p
        assert _apply_err(h, S, M) <= bar
        _, its_o, _ = O.pcg(S.A, synth.rhs(M.n, 0), lambda v: O.apply(S, v), rtol=1e-8)
        st = _pcg_its(h, M)
        assert abs(st.iterations - its_o) <= 1
    finally:
        A.destroy(h)


def test_learned_start_trains_and_is_accepted(capsys):
    """Train on subdomains of seeds 1-6, evaluate on the unseen seeds 7-8:
    the learned start is accepted, keeps the preconditioner (PCG iterations
    +-1 against the oracle, condition estimate under the bound), and the
    LOBPCG iteration counts with and without it are reported."""
    train = [_diff(10, 8, s, 1, 0.5, 60, 200) for s in range(1, 7)]
    feats, tgts = Lg.collect(train, precision=0)
    assert len(feats) >= 20
    model = Lg.ProposalModel(seed=0)
    hist = model.fit(feats, tgts, steps=300, lr=1e-3)
    assert hist[-1] < hist[0]
    cold_total = warm_total = 0
    for seed in (7, 8):
        prob = _diff(10, 8, seed, 1, 0.5, 60, 200)
        M, part, N, ov, tau = prob
        S = O.setup(M, part, N, ov, tau)
        hc, kc = _setup(prob, eig_solver=1)
        hw, kw = _setup(prob, opts=model.opts(precision=0))
        try:
            ic, iw = A.get_info(hc), A.get_info(hw)
            assert iw.lobpcg_subdomains == iw.n_partial and iw.lobpcg_fallbacks == 0
            cold_total += ic.lobpcg_iters_total
            warm_total += iw.lobpcg_iters_total
            assert _apply_err(hw, S, M) <= 1e-8
            _, its_o, _ = O.pcg(S.A, synth.rhs(M.n, 0), lambda v: O.apply(S, v), rtol=1e-8)
            st = _pcg_its(hw, M)
            assert abs(st.iterations - its_o) <= 1
            bound = O.condition_bound(O.colouring_number(S), O.splitting_constant(S), tau)
            assert st.cond_est <= bound
        finally:
            A.destroy(hc)
            A.destroy(hw)
    with capsys.disabled():
        print(f"\n[learned start] training loss {hist[0]:.3f} -> {hist[-1]:.3f}; LOBPCG iterations on unseen "
              f"subdomains: cold {cold_total}, learned {warm_total}")
    assert warm_total <= cold_total + 2


def test_feature_standardisation_kernel():
    """Column means and population standard deviations of the features come
    from the library's kernel (FP64 sums): equal to numpy's to 1e-6, and a
    constant column gets sd = 1."""
    rng = np.random.default_rng(5)
    f = (rng.standard_normal((257, A.PROP_NF)) * rng.uniform(0.1, 50, A.PROP_NF) + rng.uniform(-3, 3, A.PROP_NF))
    f[:, 7] = 2.5
    f = f.astype(np.float32)
    fd = torch.from_numpy(f).cuda()
    mean = torch.empty(A.PROP_NF, dtype=torch.float32, device="cuda")
    sd = torch.empty_like(mean)
    A.mlp_feature_stats(fd.data_ptr(), f.shape[0], mean.data_ptr(), sd.data_ptr(), stream_ptr())
    f64 = f.astype(np.float64)
    mu, s = f64.mean(axis=0), f64.std(axis=0)
    s[7] = 1.0
    assert np.allclose(mean.cpu().numpy(), mu, rtol=1e-6, atol=1e-6)
    assert np.allclose(sd.cpu().numpy(), s, rtol=1e-6, atol=1e-7)


def _c2_shaped(seed, m=24, N=16, tau=0.5):
    """The 3D channelled diffusion of the paper-scale configuration (sigma 2,
    correlation length 8, 16 channels of 1e6), 16 BFS subdomains of
    256..2048 cells, overlap 2, tau = 0.5 (partial selections)."""
    w = synth.workload_diffusion3d(m=m, N=N, lo=256, hi=2048, tau=tau, seed=seed)
    return w["A"], w["part"], w["N"], w["overlap"], w["tau"]


def test_learned_start_at_scale(capsys):
    """The learned warm start on subdomains of 740..980 owned unknowns (1.3k..2.4k
    with the overlap), mixed form: trained on 8 seeded problems (128
    subdomains), evaluated on 2 unseen seeds.  Every learned result must be
    accepted or fall back, and keep the preconditioner (PCG iterations +-1
    against the dense eigenvector path); the LOBPCG iteration counts and setup
    times with and without the network are reported, and the learned start
    may not cost more than 10% over the cold start in iterations."""
    import time
    train = [_c2_shaped(1000 + s) for s in range(8)]
    feats, tgts = Lg.collect(train, precision=1)
    assert len(feats) >= 32
    model = Lg.ProposalModel(seed=0)
    hist = model.fit(feats, tgts, steps=400, lr=1e-3)
    assert hist[-1] < hist[0]
    tot = {"cold": 0, "learned": 0}
    ms = {"cold": 0.0, "learned": 0.0, "dense": 0.0}
    for seed in (5000, 5001):
        prob = _c2_shaped(seed)
        M = prob[0]
        t0 = time.perf_counter()
        hd, kd = _setup(prob, precision=1, eig_solver=0)
        ms["dense"] += (time.perf_counter() - t0) * 1e3
        t0 = time.perf_counter()
        hc, kc = _setup(prob, precision=1, eig_solver=1)
        ms["cold"] += (time.perf_counter() - t0) * 1e3
        t0 = time.perf_counter()
        hw, kw = _setup(prob, opts=model.opts(precision=1), precision=1)
        ms["learned"] += (time.perf_counter() - t0) * 1e3
        try:
            idn, ic, iw = A.get_info(hd), A.get_info(hc), A.get_info(hw)
            assert ic.n_partial > 0 and iw.n_partial == ic.n_partial
            assert iw.lobpcg_subdomains + iw.lobpcg_fallbacks == iw.n_partial
            tot["cold"] += ic.lobpcg_iters_total
            tot["learned"] += iw.lobpcg_iters_total
            sd, sw = _pcg_its(hd, M), _pcg_its(hw, M)
            assert sw.converged == 1 and abs(sw.iterations - sd.iterations) <= 1
            assert idn.n_C == iw.n_C
        finally:
            for h in (hd, hc, hw):
                A.destroy(h)
    with capsys.disabled():
        print(f"\n[learned start at scale] {len(feats)} training subdomains, loss {hist[0]:.3f} -> {hist[-1]:.3f}; "
              f"LOBPCG iterations on unseen seeds: cold {tot['cold']}, learned {tot['learned']}; setup ms: dense "
              f"eigenvectors {ms['dense']:.0f}, cold LOBPCG {ms['cold']:.0f}, learned {ms['learned']:.0f}")
    assert tot["learned"] <= 1.1 * tot["cold"] + 2
