"""Pins of the oracle's learned-preconditioner reference (CPU only): BF16
rounding on values whose rounding is known, the SPD construction and its
e = 0 case, the hand-written backward pass against central differences, the
block-diagonal case where block-Jacobi is exact, and scale invariance of the
features."""
import numpy as np
import pytest

import oracle as orc
from oracle import precond as pc
import scenegen


def _spd(rng, n, cond=50.0):
    Q, _ = np.linalg.qr(rng.normal(size=(n, n)))
    ev = np.exp(rng.uniform(0.0, np.log(cond), size=n))
    return (Q * ev) @ Q.T


def _params(rng, scale=0.3):
    p = rng.normal(0.0, scale, size=pc.NPARAM)
    W1, b1, W2, b2, W3, b3 = pc.unpack(p)
    W1 *= 1.0 / np.sqrt(pc.FIN)
    W2 *= 1.0 / np.sqrt(pc.H)
    W3 *= 0.3 / np.sqrt(pc.H)
    return p


def test_bf16_round_known_values():
    # bfloat16 keeps 7 explicit mantissa bits: spacing 2^-7 on [1, 2)
    cases = {
        1.0: 1.0,
        1.0 + 2.0 ** -8: 1.0,                                # tie, 1.0 is even
        1.0 + 3 * 2.0 ** -8: 1.0 + 2.0 ** -6,                # tie, rounds to even
        1.0 + 2.0 ** -8 + 2.0 ** -20: 1.0 + 2.0 ** -7,       # above the tie
        -(1.0 + 2.0 ** -8 + 2.0 ** -20): -(1.0 + 2.0 ** -7),
        3.0: 3.0,
        2.0 ** -130: 2.0 ** -130,                            # a float32 subnormal that bfloat16 holds
        0.0: 0.0,
    }
    got = pc.bf16_round(np.array(list(cases.keys())))
    assert np.array_equal(got, np.array(list(cases.values())))


def test_zero_network_output_gives_block_jacobi():
    rng = np.random.default_rng(0)
    Sii = np.stack([_spd(rng, 9, 1e4) for _ in range(5)])
    M = pc.precond_blocks(np.zeros((5, 45)), Sii)
    for i in range(5):
        ref = np.linalg.inv(Sii[i])
        assert np.max(np.abs(M[i] - ref)) <= 1e-10 * np.max(np.abs(ref))


def test_blocks_are_spd_for_any_output():
    rng = np.random.default_rng(1)
    Sii = np.stack([_spd(rng, 9, 1e3) for _ in range(20)])
    e = rng.normal(0.0, 0.7, size=(20, 45))
    M = pc.precond_blocks(e, Sii)
    assert np.allclose(M, np.transpose(M, (0, 2, 1)), rtol=0, atol=1e-12 * np.abs(M).max())
    assert np.all(np.linalg.eigvalsh(M) > 0.0)


def _probe_data(rng, n=4, K=3):
    X = rng.normal(0.0, 0.5, size=(n, pc.FIN))
    A = pc.pack_lower(np.linalg.inv(np.linalg.cholesky(np.stack([_spd(rng, 9, 20.0) for _ in range(n)]))))
    Y = rng.normal(size=(n, K, 9))
    Z = rng.choice([-1.0, 1.0], size=(n, K, 9))
    return X, A, Y, Z


def test_probe_loss_grad_matches_central_differences():
    rng = np.random.default_rng(2)
    p = _params(rng)
    X, A, Y, Z = _probe_data(rng)
    loss, g = pc.probe_loss_grad(p, X, A, Y, Z)
    assert abs(loss - pc.probe_loss(p, X, A, Y, Z)) <= 1e-14 * loss
    # parameters of every layer, weights and biases
    W1, b1, W2, b2, W3, b3 = (a.size for a in pc.unpack(p))
    offs = np.cumsum([0, W1, b1, W2, b2, W3, b3])
    idx = np.concatenate([rng.choice(np.arange(offs[k], offs[k + 1]), size=6, replace=False)
                          for k in range(6)])
    h = 1e-6
    for i in idx:
        pp, pm = p.copy(), p.copy()
        pp[i] += h
        pm[i] -= h
        fd = (pc.probe_loss(pp, X, A, Y, Z) - pc.probe_loss(pm, X, A, Y, Z)) / (2 * h)
        assert abs(fd - g[i]) <= 1e-6 * max(1e-3, np.max(np.abs(g))), (i, fd, g[i])


def test_bf16_emulation_only_rounds():
    rng = np.random.default_rng(3)
    p = _params(rng)
    X, A, Y, Z = _probe_data(rng, n=16)
    e64, _ = pc.mlp_forward(p, X)
    e16, _ = pc.mlp_forward(p, X, bf16=True)
    rel = np.max(np.abs(e16 - e64)) / np.max(np.abs(e64))
    assert 1e-5 < rel < 5e-2
    l64, g64 = pc.probe_loss_grad(p, X, A, Y, Z)
    l16, g16 = pc.probe_loss_grad(p, X, A, Y, Z, bf16=True)
    assert abs(l16 - l64) <= 5e-2 * l64
    assert np.linalg.norm(g16 - g64) <= 5e-2 * np.linalg.norm(g64)


def test_block_diagonal_system_makes_block_jacobi_exact():
    """If S has no off-diagonal blocks, S_ii^{-1} is the exact inverse: at
    e = 0 every probe is reproduced, the loss and its gradient vanish."""
    rng = np.random.default_rng(4)
    n, K = 6, 4
    Sii = np.stack([_spd(rng, 9, 1e3) for _ in range(n)])
    Us = Sii + np.stack([_spd(rng, 9, 10.0) for _ in range(n)])
    X, A, D = pc.features(Sii, Us, 1e-3, np.full(n, 50))
    s = 1.0 / np.sqrt(D)
    Sh = Sii * s[:, :, None] * s[:, None, :]
    Z = rng.choice([-1.0, 1.0], size=(n, K, 9))
    Y = np.einsum("nab,nkb->nka", Sh, Z)
    p = _params(rng)
    W1, b1, W2, b2, W3, b3 = pc.unpack(p)
    W3[:] = 0.0
    b3[:] = 0.0
    loss, g = pc.probe_loss_grad(p, X, A, Y, Z)
    assert loss < 1e-24
    assert np.max(np.abs(g)) < 1e-12


def test_features_do_not_depend_on_the_scale_of_S():
    rng = np.random.default_rng(5)
    n = 4
    Sii = np.stack([_spd(rng, 9, 1e3) for _ in range(n)])
    Us = Sii + np.stack([_spd(rng, 9, 10.0) for _ in range(n)])
    X1, A1, _ = pc.features(Sii, Us, 1e-4, np.full(n, 10))
    X2, A2, _ = pc.features(1e5 * Sii, 1e5 * Us, 1e-4, np.full(n, 10))
    assert np.max(np.abs(X1 - X2)) < 1e-12
    assert np.max(np.abs(A1 - A2)) < 1e-10 * np.max(np.abs(A1))
    # scaled diagonal blocks are exactly unit on the diagonal: only their
    # off-diagonal entries are features
    assert np.all(np.abs(X1[:, :36]) < 1.0)


@pytest.mark.parametrize("huber", [0.0, 1.0])
def test_learned_solve_with_zero_network_is_block_jacobi_pcg(huber):
    sc = scenegen.arc_scene(6, 80, seed=11)
    pix = orc.pixels_from_scene(sc)
    blk = orc.assemble(sc.cams_init, sc.points_init, sc.cam_idx, sc.pt_idx, pix, huber)
    opts = orc.LMOptions(solver="pcg", pcg_tol=0.0, pcg_maxiter=12, huber_delta=huber)
    p = np.zeros(pc.NPARAM)
    dc, dp, its, rel = pc.solve_damped_learned(blk, sc.cam_idx, sc.pt_idx, 1e-3, opts, p)
    dc0, dp0, its0, rel0 = orc.solve_damped(blk, sc.cam_idx, sc.pt_idx, 1e-3, opts)
    assert its == its0
    assert np.max(np.abs(dc - dc0)) <= 1e-9 * np.max(np.abs(dc0))


def _random_spd_blocks(rng, C, coupling_scale=0.3):
    n = 9 * C
    A = rng.normal(size=(n, n))
    S = A @ A.T + n * np.eye(n)
    # weaken the coupling between cameras
    mask = np.kron(np.eye(C), np.ones((9, 9)))
    S = S * (mask + coupling_scale * (1 - mask))
    Sii = np.stack([S[9 * c:9 * c + 9, 9 * c:9 * c + 9] for c in range(C)])
    return S, Sii


def test_coupling_is_the_off_diagonal_block_row_norm_in_expectation():
    """E |(S^ z)_i - S^_ii z_i|^2 over Rademacher z is sum_{j != i} |S^_ij|_F^2:
    with many probes the estimate converges to it (1/sqrt(K) relative)."""
    rng = np.random.default_rng(5)
    C = 5
    S, Sii = _random_spd_blocks(rng, C)
    d = np.diag(S)
    Sh = S / np.sqrt(d[:, None] * d[None, :])
    exact = np.array([sum(np.sum(Sh[9 * i:9 * i + 9, 9 * j:9 * j + 9] ** 2) for j in range(C) if j != i)
                      for i in range(C)])
    est = pc.coupling(S, Sii, K=3000) ** 2
    assert np.max(np.abs(est - exact) / exact) < 0.08
    # two probes (the features' setting): the right order of magnitude
    two = pc.coupling(S, Sii) ** 2
    assert np.all(two > 0.1 * exact) and np.all(two < 10 * exact)


def test_coupling_vanishes_without_coupling_and_ignores_scales():
    rng = np.random.default_rng(6)
    C = 4
    S, Sii = _random_spd_blocks(rng, C, coupling_scale=0.0)
    # zero up to the rounding of the two products
    assert np.all(pc.coupling(S, Sii) < 1e-12)
    S, Sii = _random_spd_blocks(rng, C)
    scale = np.exp(rng.normal(size=9 * C) * 3)
    S2 = S * scale[:, None] * scale[None, :]
    Sii2 = np.stack([S2[9 * c:9 * c + 9, 9 * c:9 * c + 9] for c in range(C)])
    assert np.allclose(pc.coupling(S2, Sii2), pc.coupling(S, Sii), rtol=1e-12)


def test_splitmix64_matches_the_published_sequence():
    """SplitMix64 seeded with 0 yields 0xe220a8397b1dcdaf, 0x6e789e6aa1b965f4,
    0x06c45d188009454f (the generator's published first outputs; output n is
    the mix of n+1 golden-ratio increments, i.e. splitmix64(n * golden))."""
    golden, m64 = 0x9E3779B97F4A7C15, (1 << 64) - 1
    want = [0xE220A8397B1DCDAF, 0x6E789E6AA1B965F4, 0x06C45D188009454F]
    assert [pc.splitmix64((n * golden) & m64) for n in range(3)] == want


def test_rademacher_probes_are_balanced_signs():
    z0 = pc.rademacher(0, 1500)
    z1 = pc.rademacher(1, 1500)
    assert set(np.unique(z0)) == {-1.0, 1.0}
    assert abs(z0.mean()) < 0.03 and abs(z1.mean()) < 0.03
    # different probes are uncorrelated
    assert abs(np.mean(z0 * z1)) < 0.03
    # and neighbouring components of one probe too
    assert abs(np.mean(z0[:, :-1] * z0[:, 1:])) < 0.03
