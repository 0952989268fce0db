"""FP64 reference for the learned block-Jacobi correction (MLP preconditioner).

TEST INFRASTRUCTURE ONLY -- see the package docstring.

The paper preconditions its PCG with a diagonal (Sec. IV-C); the plain method
here uses the 9x9 block-Jacobi inverse of the reduced camera system S.  This
form adds a small MLP that maps per-camera quantities of S to an SPD
correction of that inverse.  None of it is in the paper; the readings are:

* Scaled coordinates.  D_i = diag(S_ii); S^ = D^{-1/2} S D^{-1/2}, so every
  block-diagonal entry of S^ is 1 and the quantities below do not depend on
  the units of the nine camera parameters.
* Features x_i (FIN = 96 numbers, ``features``): the 36 off-diagonal entries
  of S^_ii; the 45 entries R^_ab / sqrt((1 + R^_aa)(1 + R^_bb)) of the
  scaled point-elimination term R^ = D^{-1/2} (U*_i - S_ii) D^{-1/2} (how
  much of camera i's information its points carry, the coupling to other
  cameras through them); ln D_a minus its mean over a, / 10; log10(lambda) / 8;
  log10(1 + observations of camera i) / 4; the constant 1; the coupling of
  camera i to the other cameras, log10(1 + kappa_i) / 4 with kappa_i^2 an
  estimate of sum_{j != i} |S^_ij|_F^2 (the off-diagonal norm summary: for
  Rademacher probes z, E |(S^ z)_i - S^_ii z_i|^2 is exactly that sum; two
  probes, drawn by SplitMix64 from a counter, ``coupling``); zero padding.
* Network: h1 = relu(W1 x + b1), h2 = relu(W2 h1 + b2), e = W3 h2 + b3 with
  widths 96 -> 64 -> 64 -> 45.  Flat parameter layout W1 [64][96], b1 [64],
  W2 [64][64], b2 [64], W3 [45][64], b3 [45] (NPARAM = 13293).
* Correction: e fills a lower-triangular G (row-major lower triangle,
  t(a, b) = a (a + 1) / 2 + b): G_ab = e_t(a,b) below the diagonal,
  G_aa = exp(e_t(a,a)).  M_i = L_i^{-T} G G^T L_i^{-1} with L_i = chol(S_ii):
  SPD for every e, and e = 0 gives the block-Jacobi inverse S_ii^{-1}.
* Training loss: E_z |M S z - z|^2 with Rademacher probes, taken in the
  scaled coordinates where it separates per camera.  With K probes z^_ik and
  y^ = S^ z^ (one implicit Schur product per probe), M^_i = A_i^T G G^T A_i,
  A_i = chol(S^_ii)^{-1}: l_i = 1/(9K) sum_k |M^_i y^_ik - z^_ik|^2, and the
  loss is the mean of l_i over the cameras.
* BF16: the GPU feeds the tensor cores BF16 copies of x, W1..W3, h1, h2 and,
  going back, of dl/de, dl/dh2, dl/dh1 (accumulating in FP32).  ``bf16=True``
  rounds the same quantities (round to nearest even) so that the oracle and
  the kernels differ only by the order of FP32 accumulation.
"""
from __future__ import annotations

import numpy as np

FIN, H, FOUT = 96, 64, 45
NPARAM = H * FIN + H + H * H + H + FOUT * H + FOUT

__all__ = ["FIN", "H", "FOUT", "NPARAM", "COUPLING_PROBES", "bf16_round", "unpack", "lower_index",
           "pack_lower", "unpack_lower", "splitmix64", "rademacher", "coupling", "features", "mlp_forward",
           "g_from_e", "precond_blocks", "probe_loss", "probe_loss_grad", "solve_damped_learned"]

COUPLING_PROBES = 2
_M64 = (1 << 64) - 1


def bf16_round(x):
    """Round to the nearest bfloat16 (ties to even), returned as float64.

    bfloat16 keeps the top 16 bits of an IEEE float32: the value is first
    rounded to float32, then its low 16 bits are rounded away."""
    f = np.ascontiguousarray(np.asarray(x, dtype=np.float32))
    u = f.view(np.uint32).astype(np.uint64)
    lsb = (u >> np.uint64(16)) & np.uint64(1)
    r = ((u + np.uint64(0x7FFF) + lsb) & np.uint64(0xFFFF0000)).astype(np.uint32)
    return r.view(np.float32).astype(np.float64).reshape(np.shape(x))


def unpack(params):
    """Views of the flat parameter vector: W1, b1, W2, b2, W3, b3."""
    p = np.asarray(params, dtype=np.float64)
    assert p.shape == (NPARAM,)
    o = 0
    out = []
    for shape in ((H, FIN), (H,), (H, H), (H,), (FOUT, H), (FOUT,)):
        n = int(np.prod(shape))
        out.append(p[o:o + n].reshape(shape))
        o += n
    return out


def lower_index(a, b):
    """Position of (a, b), a >= b, in a row-major packed lower triangle."""
    return a * (a + 1) // 2 + b


def pack_lower(L):
    """[..., 9, 9] lower triangle -> [..., 45] (row-major)."""
    rows, cols = np.tril_indices(9)
    return L[..., rows, cols]


def unpack_lower(v):
    rows, cols = np.tril_indices(9)
    L = np.zeros(v.shape[:-1] + (9, 9))
    L[..., rows, cols] = v
    return L


def splitmix64(x):
    """The SplitMix64 output function of counter x (Steele, Lea and Flood,
    "Fast splittable pseudorandom number generators", OOPSLA 2014): add the
    golden-ratio increment, then two xor-shift-multiply rounds and a final
    xor-shift, all modulo 2^64."""
    z = (int(x) + 0x9E3779B97F4A7C15) & _M64
    z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & _M64
    z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & _M64
    return z ^ (z >> 31)


def rademacher(k, C):
    """Coupling probe k: [C, 9] entries +-1, entry (c, a) the sign bit of
    splitmix64(k << 40 | c << 4 | a) (1 -> -1)."""
    z = np.empty((C, 9))
    for c in range(C):
        for a in range(9):
            z[c, a] = -1.0 if splitmix64((k << 40) | (c << 4) | a) >> 63 else 1.0
    return z


def coupling(S, Sii, K=COUPLING_PROBES):
    """kappa_i: sqrt of the mean over K probes of |(S^ z)_i - S^_ii z_i|^2
    per camera, S^ = D^{-1/2} S D^{-1/2}, D = diag(S_ii): an estimate of the
    Frobenius norm of camera i's block row of S^ without its diagonal block
    (E of its square is exactly sum_{j != i} |S^_ij|_F^2).  S: the explicit
    reduced system [9C, 9C]; Sii: [C, 9, 9]; a camera with a non-positive
    diagonal gets 0."""
    Sii = np.asarray(Sii, dtype=np.float64)
    C = Sii.shape[0]
    d = np.einsum("cii->ci", Sii).reshape(-1)
    s = np.where(d > 0, 1.0 / np.sqrt(np.where(d > 0, d, 1.0)), 0.0)
    Sh = np.asarray(S, dtype=np.float64) * s[:, None] * s[None, :]
    blocks = np.stack([Sh[9 * c:9 * c + 9, 9 * c:9 * c + 9] for c in range(C)])
    acc = np.zeros(C)
    for k in range(K):
        z = rademacher(k, C)
        off = (Sh @ z.reshape(-1)).reshape(C, 9) - np.einsum("cab,cb->ca", blocks, z)
        acc += np.sum(off * off, axis=1)
    return np.sqrt(acc / K)


def features(Sii, Us, lam, nobs, kappa=None):
    """Features x [C, FIN], scaled inverse factors A = chol(S^_ii)^{-1}
    [C, 45] (packed lower) and the scales D [C, 9].

    Sii: [C, 9, 9] diagonal blocks of S; Us: [C, 9, 9] damped U*;
    nobs: [C] observations per camera; kappa: [C] coupling (``coupling``;
    None: 0).  A camera whose S_ii is not positive definite gets x = 0,
    A = 0 (it keeps the block-Jacobi fallback)."""
    Sii = np.asarray(Sii, dtype=np.float64)
    C = Sii.shape[0]
    X = np.zeros((C, FIN))
    A = np.zeros((C, 45))
    D = np.zeros((C, 9))
    iu = np.triu_indices(9, 1)
    iu0 = np.triu_indices(9)
    for i in range(C):
        d = np.diag(Sii[i]).copy()
        if not np.all(d > 0):
            continue
        s = 1.0 / np.sqrt(d)
        Sh = Sii[i] * s[:, None] * s[None, :]
        try:
            Lh = np.linalg.cholesky(Sh)
        except np.linalg.LinAlgError:
            continue
        R = (Us[i] - Sii[i]) * s[:, None] * s[None, :]
        rd = np.diag(R)
        Rn = R / np.sqrt((1.0 + rd)[:, None] * (1.0 + rd)[None, :])
        ld = np.log(d)
        X[i, 0:36] = Sh[iu]
        X[i, 36:81] = Rn[iu0]
        X[i, 81:90] = (ld - ld.mean()) / 10.0
        X[i, 90] = np.log10(lam) / 8.0
        X[i, 91] = np.log10(1.0 + nobs[i]) / 4.0
        X[i, 92] = 1.0
        X[i, 93] = 0.0 if kappa is None else np.log10(1.0 + kappa[i]) / 4.0
        A[i] = pack_lower(np.linalg.inv(Lh))
        D[i] = d
    return X, A, D


def mlp_forward(params, X, bf16=False):
    """e [n, 45] and the activations (for the backward pass)."""
    W1, b1, W2, b2, W3, b3 = unpack(params)
    rnd = bf16_round if bf16 else (lambda v: np.asarray(v, dtype=np.float64))
    x = rnd(X)
    a1 = x @ rnd(W1).T + b1
    h1 = np.maximum(a1, 0.0)
    a2 = rnd(h1) @ rnd(W2).T + b2
    h2 = np.maximum(a2, 0.0)
    e = rnd(h2) @ rnd(W3).T + b3
    return e, dict(x=x, a1=a1, h1=h1, a2=a2, h2=h2)


def g_from_e(e):
    """Lower-triangular G [..., 9, 9]: off-diagonal e, diagonal exp(e)."""
    G = unpack_lower(np.asarray(e, dtype=np.float64))
    idx = np.arange(9)
    G[..., idx, idx] = np.exp(G[..., idx, idx])
    return G


def precond_blocks(e, Sii):
    """M_i = L_i^{-T} G_i G_i^T L_i^{-1}, L_i = chol(S_ii)  [C, 9, 9]."""
    G = g_from_e(e)
    Li = np.linalg.inv(np.linalg.cholesky(np.asarray(Sii, dtype=np.float64)))
    B = np.transpose(G, (0, 2, 1)) @ Li
    return np.transpose(B, (0, 2, 1)) @ B


def _probe_terms(G, A, Y, Z):
    """Forward of the per-camera probe loss; returns the pieces the backward
    pass needs.  G, A [n, 9, 9]; Y, Z [n, K, 9]."""
    u = np.einsum("nab,nkb->nka", A, Y)       # A y
    v = np.einsum("nac,nka->nkc", G, u)       # G^T u
    w = np.einsum("nac,nkc->nka", G, v)       # G v
    m = np.einsum("nab,nka->nkb", A, w)       # A^T w
    return u, v, w, m - Z


def probe_loss(params, X, A, Y, Z, bf16=False):
    """Mean over cameras of 1/(9K) sum_k |M^_i y^_ik - z^_ik|^2."""
    e, _ = mlp_forward(params, X, bf16)
    Al = unpack_lower(np.asarray(A, dtype=np.float64))
    _, _, _, r = _probe_terms(g_from_e(e), Al, np.asarray(Y, np.float64), np.asarray(Z, np.float64))
    K = r.shape[1]
    return float(np.mean(np.sum(r * r, axis=(1, 2)) / (9.0 * K)))


def probe_loss_grad(params, X, A, Y, Z, bf16=False):
    """(loss, d loss / d params [NPARAM]) by backpropagation, written out.

    Per camera: dm = 2 r / (9 K n); w = G v gives dG += dw v^T and dv = G^T dw
    with dw = A dm; v = G^T u gives dG += u dv^T; on the diagonal
    de = dG * G (G_aa = exp(e)).  Then the three layers (relu' = 1 where the
    pre-activation is positive)."""
    W1, b1, W2, b2, W3, b3 = unpack(params)
    rnd = bf16_round if bf16 else (lambda v: np.asarray(v, dtype=np.float64))
    e, c = mlp_forward(params, X, bf16)
    n = e.shape[0]
    G = g_from_e(e)
    Al = unpack_lower(np.asarray(A, dtype=np.float64))
    Y = np.asarray(Y, np.float64)
    Z = np.asarray(Z, np.float64)
    u, v, w, r = _probe_terms(G, Al, Y, Z)
    K = r.shape[1]
    loss = float(np.mean(np.sum(r * r, axis=(1, 2)) / (9.0 * K)))
    dm = 2.0 * r / (9.0 * K * n)
    dw = np.einsum("nab,nkb->nka", Al, dm)
    dG = np.einsum("nka,nkc->nac", dw, v)
    dv = np.einsum("nac,nka->nkc", G, dw)
    dG += np.einsum("nka,nkc->nac", u, dv)
    idx = np.arange(9)
    dG[:, idx, idx] *= G[:, idx, idx]
    de = pack_lower(dG)                                   # [n, 45]
    # layer 3
    db3 = de.sum(axis=0)
    dW3 = rnd(de).T @ rnd(c["h2"])
    dh2 = (rnd(de) @ rnd(W3)) * (c["a2"] > 0.0)
    # layer 2
    db2 = dh2.sum(axis=0)
    dW2 = rnd(dh2).T @ rnd(c["h1"])
    dh1 = (rnd(dh2) @ rnd(W2)) * (c["a1"] > 0.0)
    # layer 1
    db1 = dh1.sum(axis=0)
    dW1 = rnd(dh1).T @ c["x"]
    grad = np.concatenate([dW1.ravel(), db1, dW2.ravel(), db2, dW3.ravel(), db3])
    return loss, grad


def solve_damped_learned(blk, cam_idx, pt_idx, lam, opts, params, bf16=True):
    """solve_damped (PCG) with M_i from the network instead of S_ii^{-1};
    cameras whose S_ii is not positive definite keep S_ii^{-1}."""
    from . import ba_oracle as bo
    Us = bo._ustar(blk["U"], lam, opts.diag_min, opts.diag_max)
    Vinv = bo.point_damped_inverse(blk["V"], lam, opts.diag_min, opts.diag_max)
    C = Us.shape[0]
    cam_idx = np.asarray(cam_idx)
    b = -blk["gc"] + bo.segment_sum(
        cam_idx, np.einsum("oij,oj->oi", blk["W"], np.einsum("pij,pj->pi", Vinv, blk["gp"])[pt_idx]), C)
    Sii = Us - bo.segment_sum(cam_idx, blk["W"] @ Vinv[pt_idx] @ np.transpose(blk["W"], (0, 2, 1)), C)
    nobs = np.bincount(cam_idx, minlength=C)
    S, _, _, _ = bo.schur_explicit(blk, cam_idx, pt_idx, lam, opts.diag_min, opts.diag_max)
    X, _, _ = features(Sii, Us, lam, nobs, coupling(S, Sii))
    e, _ = mlp_forward(params, X, bf16)
    M = precond_blocks(e, Sii)
    dc, its, rel = bo.pcg(lambda x: bo.schur_matvec(x, Us, Vinv, blk["W"], cam_idx, pt_idx),
                          lambda r: np.einsum("cij,cj->ci", M, r), b, opts.pcg_tol, opts.pcg_maxiter)
    dp = bo.back_substitute(dc, blk, Vinv, cam_idx, pt_idx)
    return dc, dp, its, rel
