"""Learned block-Jacobi correction on the GPU: the tensor-core network's
forward pass and loss gradient against the oracle (with the kernels' BF16
rounding emulated, and in plain FP64), the training data collection against
the oracle's explicit Schur complement, a zero network equal to
block-Jacobi, the learned PCG against the oracle's learned solve, one Adam
step, frozen-camera fallback, and what training gains on held-out scenes."""
import numpy as np
import pytest
import torch

import oracle as orc
from oracle import precond as pc
import paper_2409_12190_gb300 as ba
import scenegen
from gpu_helpers import np64

pytestmark = pytest.mark.gpu

OFFS = np.cumsum([0, 64 * 96, 64, 64 * 64, 64, 45 * 64, 45])


def _f32(a):
    return np.asarray(a, dtype=np.float32).astype(np.float64)


def _T(a):
    return torch.tensor(np.asarray(a), dtype=torch.float32, device="cuda")


def _params(rng, w3=0.3):
    p = rng.normal(0.0, 0.3, size=pc.NPARAM)
    W1, b1, W2, b2, W3, b3 = pc.unpack(p)
    W1 /= np.sqrt(pc.FIN)
    W2 /= np.sqrt(pc.H)
    W3 *= w3 / np.sqrt(pc.H)
    b3 *= w3
    return _f32(p)


def _probe_data(rng, n, K):
    X = _f32(rng.normal(0.0, 0.5, size=(n, pc.FIN)))
    B = rng.normal(size=(n, 9, 9))
    S = np.eye(9)[None] * 2.0 + 0.1 * B @ np.transpose(B, (0, 2, 1))
    A = _f32(pc.pack_lower(np.linalg.inv(np.linalg.cholesky(S))))
    Y = _f32(rng.normal(size=(n, K, 9)))
    Z = rng.choice([-1.0, 1.0], size=(n, K, 9))
    return X, A, Y, Z


@pytest.mark.parametrize("n", [1, 64, 200])
def test_mlp_forward_matches_oracle(n):
    rng = np.random.default_rng(10 + n)
    p = _params(rng)
    X, _, _, _ = _probe_data(rng, n, 1)
    E = np64(ba.mlp_forward(_T(p), _T(X)))
    E16, _ = pc.mlp_forward(p, X, bf16=True)
    E64, _ = pc.mlp_forward(p, X)
    scale = np.abs(E64).max()
    # same BF16 operands, FP32 instead of FP64 accumulation
    assert np.abs(E - E16).max() <= 2e-5 * scale
    # the BF16 rounding itself
    assert np.abs(E - E64).max() <= 5e-3 * scale


def test_mlp_loss_grad_matches_oracle():
    rng = np.random.default_rng(20)
    p = _params(rng)
    X, A, Y, Z = _probe_data(rng, 150, 3)
    loss, g = ba.mlp_loss_grad(_T(p), _T(X), _T(A), _T(Y), _T(Z))
    g = np64(g)
    l16, g16 = pc.probe_loss_grad(p, X, A, Y, Z, bf16=True)
    l64, g64 = pc.probe_loss_grad(p, X, A, Y, Z)
    assert abs(loss - l16) <= 1e-6 * l16
    assert abs(loss - l64) <= 5e-3 * l64
    for k in range(6):  # every weight and bias block
        a, b = OFFS[k], OFFS[k + 1]
        assert np.linalg.norm(g[a:b] - g16[a:b]) <= 1e-5 * np.linalg.norm(g16[a:b]), k
        # BF16 rounding of the operands of three chained layers (2^-9 each)
        assert np.linalg.norm(g[a:b] - g64[a:b]) <= 6e-2 * np.linalg.norm(g64[a:b]), k


def test_adam_step_uses_the_gradient():
    rng = np.random.default_rng(21)
    p = _params(rng)
    X, A, Y, Z = _probe_data(rng, 128, 2)
    pt = _T(p)
    m = torch.zeros_like(pt)
    v = torch.zeros_like(pt)
    lr = 1e-3
    hist = ba.mlp_train(pt, m, v, _T(X), _T(A), _T(Y), _T(Z), epochs=1, batch=128, lr=lr)
    _, g16 = pc.probe_loss_grad(p, X, A, Y, Z, bf16=True)
    # first bias-corrected Adam step: m^ = g, v^ = g^2  ->  -lr g / (|g| + eps)
    ref = p - lr * g16 / (np.abs(g16) + 1e-8)
    big = np.abs(g16) > 1e-4 * np.abs(g16).max()
    assert np.max(np.abs(np64(pt) - ref)[big]) <= 1e-3 * lr
    assert len(hist) == 1 and hist[0] > 0.0


def test_learn_collect_matches_oracle():
    rng = np.random.default_rng(22)
    sc = scenegen.arc_scene(8, 200, seed=3)
    pix = orc.pixels_from_scene(sc)
    K, lam = 4, 1e-3
    zh = rng.choice([-1.0, 1.0], size=(sc.C, K, 9))
    with ba.Problem(sc.cams_init, sc.points_init, sc.cam_idx, sc.pt_idx, pix, ba.Options(precision="f64")) as prob:
        X, A, Y = (np64(t) for t in prob.learn_collect(lam, torch.tensor(zh)))
    blk = orc.assemble(sc.cams_init, sc.points_init, sc.cam_idx, sc.pt_idx, pix)
    S, _, Us, _ = orc.schur_explicit(blk, sc.cam_idx, sc.pt_idx, lam)
    Sii = np.stack([S[9 * i:9 * i + 9, 9 * i:9 * i + 9] for i in range(sc.C)])
    # the coupling feature: the same SplitMix64 probes through the explicit S
    Xo, Ao, Do = pc.features(Sii, Us, lam, np.bincount(sc.cam_idx, minlength=sc.C), pc.coupling(S, Sii))
    assert np.all(Xo[:, 93] > 0.0)
    s = 1.0 / np.sqrt(Do.reshape(-1))
    Sh = S * s[:, None] * s[None, :]
    # y^ = S^ z^ with the explicit S of the oracle, probe by probe
    Yo = np.einsum("ab,kb->ka", Sh, zh.transpose(1, 0, 2).reshape(K, -1)).reshape(K, sc.C, 9).transpose(1, 0, 2)
    # outputs are FP32
    assert np.abs(X - Xo).max() <= 1e-6
    assert np.abs(A - Ao).max() <= 1e-6 * np.abs(Ao).max()
    assert np.abs(Y - Yo).max() <= 1e-6 * np.abs(Yo).max()


def test_zero_network_is_block_jacobi():
    sc = scenegen.ring_scene(60, 3000, seed=5, view_p=1.0 / 5.7)
    pix = orc.pixels_from_scene(sc)
    o = ba.Options(precision="f64", pcg_maxiter=200, pcg_tol=1e-8)
    with ba.Problem(sc.cams_init, sc.points_init, sc.cam_idx, sc.pt_idx, pix, o) as pr:
        dc0, _, it0, _ = pr.damped_solve(1e-4, 200, 1e-8)
        pr.solve(4)
        st0 = pr.stats()
        pr.set_params(torch.from_numpy(sc.cams_init), torch.from_numpy(sc.points_init))
        pr.set_lambda(1e-4)
        pr.set_preconditioner(ba.mlp_init(0))
        dc1, _, it1, _ = pr.damped_solve(1e-4, 200, 1e-8)
        pr.solve(4)
        st1 = pr.stats()[-4:]
    assert it0 == it1
    assert float((dc1 - dc0).abs().max()) <= 1e-10 * float(dc0.abs().max())
    for a, b in zip(st0, st1):
        assert a["pcg_iters"] == b["pcg_iters"] and a["accepted"] == b["accepted"]
        assert abs(a["cost_trial"] - b["cost_trial"]) <= 1e-10 * a["cost"]


def test_learned_pcg_matches_oracle_learned_solve():
    rng = np.random.default_rng(23)
    sc = scenegen.arc_scene(10, 300, seed=12)
    pix = orc.pixels_from_scene(sc)
    p = _params(rng, w3=0.2)
    lam, iters = 1e-3, 10
    with ba.Problem(sc.cams_init, sc.points_init, sc.cam_idx, sc.pt_idx, pix, ba.Options(precision="f64")) as pr:
        pr.set_preconditioner(torch.tensor(p, dtype=torch.float32))
        dc, _, its, _ = pr.damped_solve(lam, iters, 0.0)
    blk = orc.assemble(sc.cams_init, sc.points_init, sc.cam_idx, sc.pt_idx, pix)
    opts = orc.LMOptions(solver="pcg", pcg_tol=0.0, pcg_maxiter=iters)
    dco, _, itso, _ = pc.solve_damped_learned(blk, sc.cam_idx, sc.pt_idx, lam, opts, p, bf16=True)
    dcb, _, _, _ = orc.solve_damped(blk, sc.cam_idx, sc.pt_idx, lam, opts)
    assert its == itso == iters
    err = np.abs(np64(dc) - dco).max() / np.abs(dco).max()
    # the network changed the iterate (it is not block-Jacobi) ...
    assert np.abs(dcb - dco).max() / np.abs(dco).max() > 100 * err
    # ... and the GPU follows the oracle's learned solve
    assert err <= 1e-6


def test_frozen_cameras_keep_block_jacobi():
    sc = scenegen.arc_scene(8, 200, seed=13)
    pix = orc.pixels_from_scene(sc)
    p = _params(np.random.default_rng(24), w3=0.2)
    with ba.Problem(sc.cams_init, sc.points_init, sc.cam_idx, sc.pt_idx, pix,
                    ba.Options(precision="f64", pcg_maxiter=20)) as pr:
        pr.set_fixed(torch.from_numpy(orc.gauge_mask(sc.C)))
        pr.set_preconditioner(torch.tensor(p, dtype=torch.float32))
        pr.solve(2)
        st = pr.stats()
    # cameras 0 and 1 have frozen parameters: their blocks stay block-Jacobi
    assert all(t["precond_fallbacks"] == 2 for t in st)
    assert st[0]["accepted"]


def _problem(scene, prec="f32"):
    pix = torch.tensor(orc.pixels_from_scene(scene))
    return ba.Problem(scene.cams_init, scene.points_init, scene.cam_idx, scene.pt_idx, pix,
                      ba.Options(precision=prec, pcg_maxiter=50, pcg_tol=1e-4))


def test_slow_probes_are_scaled_truncated_pcg_errors():
    sc = scenegen.ring_scene(40, 2000, seed=9, view_p=1.0 / 5.7)
    with _problem(sc, "f64") as pr:
        lam = 1e-4
        z = np64(pr.learn_slow_probes(lam, (5, 15), 400, 1e-12))
        _, _, _, D = pr.learn_collect(lam, torch.zeros((sc.C, 0, 9)), scales=True)
        xr, _, _, _ = pr.damped_solve(lam, 400, 1e-12)
        x5, _, _, _ = pr.damped_solve(lam, 5, 0.0)
    e = (np64(xr) - np64(x5)) * np.sqrt(np64(D))
    e /= np.sqrt(np.mean(e * e))
    assert np.abs(z[:, 0, :] - e).max() <= 1e-5 * np.abs(e).max()
    assert abs(np.sqrt(np.mean(z[:, 1, :] ** 2)) - 1.0) < 1e-6


def test_training_lowers_held_out_probe_loss_and_keeps_pcg_near_block_jacobi():
    """Trained on ring scenes (Rademacher plus slow-mode probes), the network
    lowers the held-out probe loss below block-Jacobi's (its zero output).
    The slow-mode probes, which no block-diagonal M fits, keep that loss
    high. PCG iterations to 1e-6 on six held-out systems (three 300-camera
    rings, lambda = 1e-4 and 1e-3, FP64) stay near block-Jacobi's but do
    not drop reliably. Measured over training seeds 0-3, per system the
    learned count is 0.85 to 1.17 times block-Jacobi's and the total is
    0.97 to 1.02 times. The test bounds the total at 1.05 and each system
    at 1.25."""
    from paper_2409_12190_gb300 import learned
    rng = np.random.default_rng(25)
    samples = []
    for i, C in enumerate(rng.integers(60, 200, size=10)):
        with _problem(scenegen.ring_scene(int(C), 100 * int(C), seed=1000 + i, view_p=1.0 / 5.7)) as pr:
            samples.append(learned.collect(pr, seed=i))
    with _problem(scenegen.ring_scene(300, 30000, seed=2000, view_p=1.0 / 5.7)) as pr:
        held = learned.collect(pr, states=(0, 2), seed=99)
    l_bj = learned.held_out_loss(ba.mlp_init(0), held)
    params, hist = learned.train(samples, epochs=100, lr=2e-3)
    l_tr = learned.held_out_loss(params, held)
    assert hist[-1] < hist[0]
    assert l_tr <= 0.98 * l_bj, (l_bj, l_tr)
    its = []
    for seed in (2001, 2002, 2003):
        sc = scenegen.ring_scene(300, 30000, seed=seed, view_p=1.0 / 5.7)
        with _problem(sc, "f64") as pr:
            for lam in (1e-4, 1e-3):
                pr.set_preconditioner(None)
                _, _, it_bj, _ = pr.damped_solve(lam, 1000, 1e-6)
                pr.set_preconditioner(params)
                _, _, it_l, _ = pr.damped_solve(lam, 1000, 1e-6)
                its.append((it_bj, it_l))
    tot_bj, tot_l = sum(i[0] for i in its), sum(i[1] for i in its)
    print(f"held-out probe loss {l_bj:.4f} -> {l_tr:.4f}; PCG iterations to 1e-6 "
          f"(block-Jacobi, learned): {its}, total ratio {tot_l / tot_bj:.3f}")
    assert tot_l <= 1.05 * tot_bj
    assert all(l <= 1.25 * b for b, l in its), its
