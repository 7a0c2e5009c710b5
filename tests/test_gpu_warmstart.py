"""GPU parity of the learned warm start: network forward, gradient and Adam step against the
FP64 oracle, the snapshot basis against the oracle's randomized subspace iteration, the
guarded PCG, and an end-to-end check that the trained network saves PCG iterations.

Tolerances. The network keeps BF16 weights (the oracle is given exactly those values) and
FP32 activations with FP32 accumulation, so a forward value or gradient entry carries at most
~n u_32 relative error, n the longest chain of roundings (depth x (width + batch) <= 3 x 300
here): 900 x 6e-8 = 5e-5 of the largest entry; the tests use 1e-4. The basis is built from
FP32 products: its rows move by ~kappa(Omega^T Y) u_32 from the FP64 oracle's; the spectra
used keep kappa <= 30, so 1e-4 is ~50x that estimate.
"""
import math

import numpy as np
import pytest

from oracle import warmstart as W
from tests._common import sample_initial, sample_potential
from inputs import harmonic_potential, wavepacket_factors, wavepacket_params

pytestmark = pytest.mark.gpu


def _torch():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    return torch


def _bf16(x):
    """Round to the nearest bfloat16 (ties to even), returned as float64."""
    f = np.asarray(x, dtype=np.float32).view(np.uint32).astype(np.uint64)
    f = (f + 0x7FFF + ((f >> 16) & 1)) & 0xFFFF0000
    return f.astype(np.uint32).view(np.float32).astype(np.float64)


def _net(sizes, max_batch, seed=1):
    import paper_2311_18461_gb300 as P
    torch = _torch()
    w = P.stst_ws_create(sizes, max_batch, seed, torch.cuda.current_stream())
    n = P.stst_ws_num_params(w)
    assert n == W.n_params(sizes)
    theta = torch.empty(n, dtype=torch.float32, device="cuda")
    P.stst_ws_get_params(w, theta)
    return w, theta.cpu().numpy().astype(np.float64)


def _rel(a, b):
    return float(np.abs(np.asarray(a) - np.asarray(b)).max() / max(np.abs(np.asarray(b)).max(), 1e-300))


@pytest.mark.parametrize("sizes,B", [([7, 64, 64, 48], 37), ([5, 100, 3], 1), ([33, 70, 50], 8),
                                     ([9, 130, 70, 65, 20], 256)])
def test_forward_matches_oracle(sizes, B):
    import paper_2311_18461_gb300 as P
    torch = _torch()
    w, theta = _net(sizes, 256)
    try:
        X = np.random.default_rng(0).standard_normal((B, sizes[0])).astype(np.float32)
        Y = torch.empty((B, sizes[-1]), dtype=torch.float32, device="cuda")
        P.stst_ws_forward(w, torch.tensor(X, device="cuda"), B, Y)
        torch.cuda.synchronize()
        ref, _ = W.forward(theta, sizes, X.astype(np.float64))
        assert _rel(Y.cpu().numpy(), ref) < 1e-4
    finally:
        P.stst_ws_destroy(w)


def test_forward_output_scale_and_accumulation():
    import paper_2311_18461_gb300 as P
    torch = _torch()
    sizes = [6, 40, 12]
    for B in (3, 20):  # the one-warp-per-row path and the tiled path
        w, theta = _net(sizes, 32)
        try:
            rng = np.random.default_rng(B)
            X = rng.standard_normal((B, 6)).astype(np.float32)
            Y0 = rng.standard_normal((B, 12)).astype(np.float32)
            sc = rng.uniform(0.5, 2.0, size=12).astype(np.float32)
            P.stst_ws_set_output_scale(w, torch.tensor(sc, device="cuda"))
            Y = torch.tensor(Y0, device="cuda")
            P.stst_ws_forward(w, torch.tensor(X, device="cuda"), B, Y, 0.5)
            ref = W.forward(theta, sizes, X.astype(np.float64))[0] * sc + 0.5 * Y0
            assert _rel(Y.cpu().numpy(), ref) < 1e-5
            P.stst_ws_set_output_scale(w, None)
            P.stst_ws_forward(w, torch.tensor(X, device="cuda"), B, Y)
            assert _rel(Y.cpu().numpy(), W.forward(theta, sizes, X.astype(np.float64))[0]) < 1e-5
        finally:
            P.stst_ws_destroy(w)


@pytest.mark.parametrize("sizes,rows,B", [([7, 64, 64, 48], 90, 37), ([5, 300, 300, 256], 400, 256)])
def test_gradient_matches_oracle(sizes, rows, B):
    import paper_2311_18461_gb300 as P
    torch = _torch()
    w, theta = _net(sizes, 256)
    try:
        rng = np.random.default_rng(1)
        X = rng.standard_normal((rows, sizes[0])).astype(np.float32)
        T = rng.standard_normal((rows, sizes[-1])).astype(np.float32)
        wt = rng.uniform(0.2, 2.0, size=rows).astype(np.float32)
        idx = rng.permutation(rows)[:B].astype(np.int32)
        g = torch.empty(len(theta), dtype=torch.float32, device="cuda")
        loss = P.stst_ws_grad(w, torch.tensor(X, device="cuda"), torch.tensor(T, device="cuda"),
                              torch.tensor(wt, device="cuda"), torch.tensor(idx, device="cuda"), B, g)
        Lr, gr = W.loss_grad(theta, sizes, X[idx].astype(np.float64), T[idx].astype(np.float64),
                             wt[idx].astype(np.float64))
        assert abs(loss - Lr) <= 1e-4 * abs(Lr)
        gg = g.cpu().numpy()
        for (ws, _), bs in W.layer_slices(sizes):
            assert _rel(gg[ws], gr[ws]) < 1e-4
            assert _rel(gg[bs], gr[bs]) < 1e-4
    finally:
        P.stst_ws_destroy(w)


def test_adam_step_matches_oracle():
    import paper_2311_18461_gb300 as P
    torch = _torch()
    sizes = [6, 48, 32, 10]
    w, _ = _net(sizes, 64)
    try:
        rng = np.random.default_rng(2)
        theta = np.zeros(W.n_params(sizes))
        isw = np.zeros(len(theta), dtype=bool)
        for (ws, shape), bs in W.layer_slices(sizes):
            theta[ws] = _bf16(rng.standard_normal(shape[0] * shape[1]) / math.sqrt(shape[1]))
            theta[bs] = rng.standard_normal(shape[0]).astype(np.float32) * 0.1
            isw[ws] = True
        P.stst_ws_set_params(w, torch.tensor(theta, dtype=torch.float32, device="cuda"))
        X = rng.standard_normal((40, sizes[0])).astype(np.float32)
        T = rng.standard_normal((40, sizes[-1])).astype(np.float32)
        lr = 2.0 ** -9
        P.stst_ws_train_step(w, torch.tensor(X, device="cuda"), torch.tensor(T, device="cuda"), None, None, 40, lr)
        out = torch.empty(len(theta), dtype=torch.float32, device="cuda")
        P.stst_ws_get_params(w, out)
        got = out.cpu().numpy().astype(np.float64)
        _, g = W.loss_grad(theta, sizes, X.astype(np.float64), T.astype(np.float64))
        ref, _, _ = W.adam(theta, g, np.zeros_like(g), np.zeros_like(g), 1, lr)
        # weights: the BF16 copy of the FP32 master (one BF16 ulp = 2^-7 relative at most);
        # entries with |g| near eps move by less than lr and are compared the same way
        refw = ref[isw]
        assert np.all(np.abs(got[isw] - refw) <= 2.0 ** -7 * np.abs(refw) + 1e-6)
        assert _rel(got[~isw], ref[~isw]) < 1e-5
        moved = np.abs(got[isw] - theta[isw]) > 0
        assert moved.mean() > 0.5  # the step is visible through the BF16 rounding
    finally:
        P.stst_ws_destroy(w)


def test_training_fits_a_smooth_map():
    import paper_2311_18461_gb300 as P
    torch = _torch()
    sizes = [3, 64, 64, 4]
    w, _ = _net(sizes, 128)
    try:
        rng = np.random.default_rng(3)
        X = rng.uniform(-1, 1, size=(512, 3)).astype(np.float32)
        T = np.stack([np.sin(X[:, 0] + 0.5 * j) * np.cos(0.5 * X[:, 1] - 0.3 * j * X[:, 2]) for j in range(4)], 1)
        Xd = torch.tensor(X, device="cuda")
        Td = torch.tensor(T.astype(np.float32), device="cuda")
        first = P.stst_ws_grad(w, Xd, Td, None, None, 128, None)
        for k in range(1500):
            idx = torch.tensor(rng.permutation(512)[:128].astype(np.int32), device="cuda")
            P.stst_ws_train_step(w, Xd, Td, None, idx, 128, 3e-3 * (1 - k / 1500) + 1e-5)
        last = P.stst_ws_grad(w, Xd, Td, None, None, 128, None)
        assert last < first / 50
    finally:
        P.stst_ws_destroy(w)


def _snapshots(n, m, decay, seed, rank=None):
    rng = np.random.default_rng(seed)
    r = rank or min(n, m)
    U, _ = np.linalg.qr(rng.standard_normal((n, r)))
    V, _ = np.linalg.qr(rng.standard_normal((m, r)))
    s = decay ** np.arange(r)
    return (U * s) @ V.T


@pytest.mark.parametrize("n,m,K,q", [(96, 1000, 16, 0), (96, 1000, 16, 1), (300, 4100, 64, 1), (64, 777, 64, 0)])
def test_pod_basis_matches_oracle(n, m, K, q):
    import paper_2311_18461_gb300 as P
    torch = _torch()
    Y = _snapshots(n, m, 0.97, seed=n + K)
    Om = np.random.default_rng(7).standard_normal((n, K)).astype(np.float32)
    Q = torch.empty((K, m), dtype=torch.float32, device="cuda")
    P.stst_pod_basis(torch.tensor(Y, device="cuda"), n, m, torch.tensor(Om, device="cuda"), K, q, Q)
    Qg = Q.cpu().numpy().astype(np.float64)
    ref = W.range_basis(Y, Om.astype(np.float64), q)
    assert np.abs(Qg @ Qg.T - np.eye(K)).max() < 1e-5
    assert _rel(Qg, ref) < 1e-4


def test_pod_basis_captures_a_rank_K_set_exactly_and_flags_a_deficient_one():
    import paper_2311_18461_gb300 as P
    torch = _torch()
    n, m, K = 80, 2000, 12
    rng = np.random.default_rng(8)
    Y = rng.standard_normal((n, K)) @ rng.standard_normal((K, m))
    Om = torch.tensor(rng.standard_normal((n, K)).astype(np.float32), device="cuda")
    Q = torch.empty((K, m), dtype=torch.float32, device="cuda")
    P.stst_pod_basis(torch.tensor(Y, device="cuda"), n, m, Om, K, 1, Q)
    Qg = Q.cpu().numpy().astype(np.float64)
    assert np.linalg.norm(Y - Y @ Qg.T @ Qg) <= 1e-5 * np.linalg.norm(Y)
    # K + 4 requested directions from a rank-K set: the Gram matrix is singular
    Om2 = torch.tensor(rng.standard_normal((n, K + 4)).astype(np.float32), device="cuda")
    Q2 = torch.empty((K + 4, m), dtype=torch.float32, device="cuda")
    Yr = torch.tensor(np.repeat(Y[:1], n, axis=0), device="cuda")  # rank 1
    assert P.stst_pod_basis(Yr, n, m, Om2, K + 4, 0, Q2) == 3  # STST_NOT_HPD
    with pytest.raises(P.StstError):
        P.stst_pod_basis(Yr, n, m, Om2, n + 1, 0, Q2)  # K > n


@pytest.mark.parametrize("n", [1, 5, 16, 70])
def test_pod_project_and_expand_match_definitions(n):
    import paper_2311_18461_gb300 as P
    torch = _torch()
    m, K = 13002, 40
    rng = np.random.default_rng(9 + n)
    Y = rng.standard_normal((n, m))
    Q = np.ascontiguousarray(np.linalg.qr(rng.standard_normal((m, K)))[0].T.astype(np.float32))
    C = torch.empty((n, K), dtype=torch.float32, device="cuda")
    Qd = torch.tensor(Q, device="cuda")
    P.stst_pod_project(torch.tensor(Y, device="cuda"), n, m, Qd, K, C)
    assert _rel(C.cpu().numpy(), Y @ Q.T.astype(np.float64)) < 1e-6
    Cn = rng.standard_normal((n, K)).astype(np.float32)
    phase = rng.uniform(0, 2 * np.pi, size=n)
    X0 = rng.standard_normal((n, m))
    X = torch.tensor(X0, device="cuda")
    P.stst_pod_expand(Qd, K, m, torch.tensor(Cn, device="cuda"), n, 0.5, -2.0, torch.tensor(phase, device="cuda"), X)
    ref = 0.5 * Cn.astype(np.float64) @ Q.astype(np.float64) - 2.0 * X0
    refc = (ref[:, 0::2] + 1j * ref[:, 1::2]) * np.exp(1j * phase)[:, None]
    got = X.cpu().numpy()
    assert _rel(got[:, 0::2] + 1j * got[:, 1::2], refc) < 1e-6


def _small_problem(prec=1):
    import paper_2311_18461_gb300 as P
    prob = P.Problem(2, [10, 10, 10], 3, prec_mode=prec)
    V = harmonic_potential(2)
    prob.set_potential(sample_potential(prob, V), len(V))
    prob.build_fd()
    return prob


def _wavepacket_rhs(prob, par):
    return prob.rhs(u0_qp=sample_initial(prob, wavepacket_factors(par)))


def test_guarded_pcg_keeps_good_and_rejects_bad_guesses():
    torch = _torch()
    prob = _small_problem()
    par = wavepacket_params(np.random.default_rng(11), 2)
    f = _wavepacket_rhs(prob, par)
    x, s, it0, rr = prob.pcg(f, tol=1e-10)
    assert s == 0
    good = x * (1 + 1e-5 * torch.randn_like(x.real))
    _, s, it1, rr1, used = prob.pcg_guarded(f, good.clone(), tol=1e-10)
    assert s == 0 and used == 1 and it1 < it0 and rr1 <= 1e-10
    bad = 1e3 * torch.randn_like(x)
    xb, s, it2, rr2, used = prob.pcg_guarded(f, bad, tol=1e-10)
    assert s == 0 and used == 0 and it2 == it0
    assert torch.abs(xb - x).max().item() <= 1e-12 * torch.abs(x).max().item()
    nan = torch.full_like(x, float("nan"))
    _, s, it3, _, used = prob.pcg_guarded(f, nan, tol=1e-10)
    assert s == 0 and used == 0 and it3 == it0
    prob.close()


def test_trained_warm_start_saves_iterations():
    """Small version of the learned-warm-start workload: train on 400 solves, evaluate on 12 new ones."""
    from paper_2311_18461_gb300.warmstart import WarmStart
    torch = _torch()
    prob = _small_problem()
    rng = np.random.default_rng(12)
    train = [wavepacket_params(rng, 2) for _ in range(400)]
    ws = WarmStart(prob, K_in=200, K_out=200, hidden=(), stages=2, max_batch=128, seed=3)
    ws.collect([lambda par=par: sample_initial(prob, wavepacket_factors(par)) for par in train])
    ws.fit(power_its=1, seed=4)
    hist = ws.train(3000, batch=128, lr0=2e-3, lr1=1e-6, seed=5, log_every=500)
    first_stage = [loss for stage, _, loss in hist if stage == 0]
    assert first_stage[-1] < first_stage[0] / 100
    cold, warm, err = [], [], []
    test_rng = np.random.default_rng(99)
    for _ in range(12):
        par = wavepacket_params(test_rng, 2)
        f, c0 = prob.rhs(u0_qp=sample_initial(prob, wavepacket_factors(par)), want_c0=True)
        xc, s, itc, _ = prob.pcg(f, tol=1e-8)
        assert s == 0
        x0 = ws.predict(c0)[0].clone()
        e0 = (torch.linalg.vector_norm(x0 - xc) / torch.linalg.vector_norm(xc)).item()
        xw, s, itw, rr, used = ws.solve(f, x0, tol=1e-8)
        assert s == 0 and rr <= 1e-8 and used == 1
        cold.append(itc)
        warm.append(itw)
        err.append((e0, (torch.linalg.vector_norm(xw - xc) / torch.linalg.vector_norm(xc)).item()))
    ws.close()
    prob.close()
    # the arbiter: the same tolerance is met from the learned start in fewer iterations
    assert np.mean(warm) < np.mean(cold) - 1.0, (cold, warm, err)
    assert max(e[1] for e in err) < 1e-5


# ---- training-data preparation on the device -------------------------------------------------------
# Inputs are FP32; the device forms the Gram matrix, the Cholesky factor and its inverse in FP64 (as the
# oracle does) and rounds the whitened features and the rotated basis to FP32 after FP64 products:
# ~kappa(F) u_32 relative, kappa(F) <= 30 here, so 1e-5. The scalings are FP64 sums of FP32 squares
# (1e-12 on so) rounded to FP32 (1e-6 on the scaled targets and weights).
def test_whitening_matches_oracle():
    import paper_2311_18461_gb300 as P
    torch = _torch()
    rng = np.random.default_rng(21)
    n, K, m = 700, 40, 300
    F = (rng.standard_normal((n, K)) @ (rng.standard_normal((K, K)) * np.logspace(0, -1, K)).T).astype(np.float32)
    Q = rng.standard_normal((K, m)).astype(np.float32)
    Fd, Qd = torch.tensor(F, device="cuda"), torch.tensor(Q, device="cuda")
    Fw = torch.empty_like(Fd)
    P.stst_ws_whiten(Fd, n, K, Fw, Qd, m)
    Wm, Fw_ref = W.whiten(F.astype(np.float64))
    rel = lambda a, b: np.abs(a - b).max() / np.abs(b).max()
    assert rel(Fw.cpu().numpy(), Fw_ref) < 1e-5
    assert rel(Qd.cpu().numpy(), Wm.T @ Q.astype(np.float64)) < 1e-5
    cov = Fw.cpu().numpy().astype(np.float64)
    assert np.abs(cov.T @ cov / n - np.eye(K)).max() < 1e-4


def test_target_scaling_and_cascade_match_oracle():
    import paper_2311_18461_gb300 as P
    torch = _torch()
    rng = np.random.default_rng(22)
    n, K = 500, 33
    T = (rng.standard_normal((n, K)) * np.logspace(0, 2, K)).astype(np.float32)
    Td = torch.tensor(T, device="cuda")
    Ts = torch.empty_like(Td)
    so = torch.empty(K, dtype=torch.float64, device="cuda")
    w = torch.empty(n, dtype=torch.float32, device="cuda")
    P.stst_ws_target_scale(Td, n, K, Ts, so, w)
    so_r, Ts_r, w_r = W.target_scaling(T.astype(np.float64))
    assert np.abs(so.cpu().numpy() / so_r - 1).max() < 1e-12
    assert np.abs(Ts.cpu().numpy() - Ts_r).max() / np.abs(Ts_r).max() < 1e-6
    assert np.abs(w.cpu().numpy() / w_r - 1).max() < 1e-6
    # two stages: the first fits the scaled targets as they are, the second the error a prediction left
    resid = torch.empty((n, K), dtype=torch.float64, device="cuda")
    scale = torch.empty(K, dtype=torch.float64, device="cuda")
    tgt = torch.empty((n, K), dtype=torch.float32, device="cuda")
    osc = torch.empty(K, dtype=torch.float32, device="cuda")
    P.stst_ws_cascade(Ts, None, None, resid, n, K, scale, tgt, so, osc)
    r0, s0, t0 = W.cascade_stage(None, T0=Ts.cpu().numpy().astype(np.float64))
    assert np.array_equal(scale.cpu().numpy(), s0) and np.abs(tgt.cpu().numpy() - t0).max() == 0
    assert np.abs(osc.cpu().numpy() / so_r - 1).max() < 1e-6
    Y = (Ts.cpu().numpy() + 1e-2 * rng.standard_normal((n, K))).astype(np.float32)  # a stage's prediction
    Yd = torch.tensor(Y, device="cuda")
    scale1 = torch.empty_like(scale)
    P.stst_ws_cascade(None, Yd, scale, resid, n, K, scale1, tgt, so, osc)
    r1, s1, t1 = W.cascade_stage(r0, Y=Y.astype(np.float64), scale_prev=s0)
    assert np.abs(resid.cpu().numpy() - r1).max() / np.abs(r1).max() < 1e-12
    assert np.abs(scale1.cpu().numpy() / s1 - 1).max() < 1e-12
    assert np.abs(tgt.cpu().numpy() - t1).max() / np.abs(t1).max() < 1e-6
    assert np.abs(osc.cpu().numpy() / (so_r * s1) - 1).max() < 1e-6
