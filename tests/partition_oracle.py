"""The LM iteration of a point-partitioned problem, written with the oracle's
pieces (test code only).

Each part holds some points with all their observations and every camera.
Everything that sums over observations is computed over the part and then
summed over the parts by ``allreduce`` -- at the same six places where the
library exchanges: U and gc of the linearisation, the Schur pass's
per-camera sums (b and the block-Jacobi blocks), the pass-B sum of every PCG
iteration, and the trial's cost, gp . dp and model term (and the starting
cost).  Everything else (the PCG vectors and dot products, the decision,
lambda) is computed identically in every part.  With one part this is the
oracle's ``lm``; with several it must reproduce it up to the summation
order."""
import numpy as np

import oracle as orc
from oracle.ba_oracle import _ustar, segment_sum


def part_lm(cams0, points0, cam_idx, pt_idx, pixels, iters, opts, allreduce):
    """LM trials of one part (points0 / pt_idx / pixels: this part's,
    cam_idx: its observations' cameras, cams0: every camera).  allreduce(a)
    returns the sum of the array a over all parts.  Returns (cams, the
    part's points, trace)."""
    cams = np.array(cams0, dtype=np.float64, copy=True)
    points = np.array(points0, dtype=np.float64, copy=True)
    C = cams.shape[0]
    delta = opts.huber_delta
    lam = opts.lambda0
    F = float(allreduce(np.array([orc.cost(cams, points, cam_idx, pt_idx, pixels, delta)]))[0])
    blk = None
    trace = []
    for _ in range(iters):
        if blk is None:
            blk = orc.assemble(cams, points, cam_idx, pt_idx, pixels, delta)
            U = allreduce(blk["U"])
            gc = allreduce(blk["gc"])
        W = blk["W"]
        Us = _ustar(U, lam, opts.diag_min, opts.diag_max)
        Vinv = orc.point_damped_inverse(blk["V"], lam, opts.diag_min, opts.diag_max)
        y = np.einsum("pij,pj->pi", Vinv, blk["gp"])
        b = -gc + allreduce(segment_sum(cam_idx, np.einsum("oij,oj->oi", W, y[pt_idx]), C))
        Sii = Us - allreduce(segment_sum(cam_idx, W @ Vinv[pt_idx] @ np.transpose(W, (0, 2, 1)), C))
        M = np.linalg.inv(Sii)

        def matvec(x):
            z = segment_sum(pt_idx, np.einsum("oij,oi->oj", W, x[cam_idx]), points.shape[0])
            t = np.einsum("pij,pj->pi", Vinv, z)
            return np.einsum("cij,cj->ci", Us, x) - \
                allreduce(segment_sum(cam_idx, np.einsum("oij,oj->oi", W, t[pt_idx]), C))

        dc, its, rel = orc.pcg(matvec, lambda r: np.einsum("cij,cj->ci", M, r), b, opts.pcg_tol,
                               opts.pcg_maxiter)
        dp = orc.back_substitute(dc, blk, Vinv, cam_idx, pt_idx)
        cams_t = cams + dc
        points_t = points + dp
        JD = np.einsum("oai,oi->oa", blk["Jc"], dc[cam_idx]) + np.einsum("oai,oi->oa", blk["Jp"], dp[pt_idx])
        sums = allreduce(np.array([orc.cost(cams_t, points_t, cam_idx, pt_idx, pixels, delta),
                                   float(np.sum(blk["gp"] * dp)),
                                   float(np.sum(blk["w"] * np.sum(JD * JD, axis=1)))]))
        Ft = float(sums[0])
        dL = -(float(np.sum(gc * dc)) + float(sums[1])) - 0.5 * float(sums[2])
        rho = (F - Ft) / dL if dL != 0.0 else float("nan")
        accept = bool(np.isfinite(Ft) and dL > 0.0 and Ft < F)
        trace.append(dict(cost=F, cost_trial=Ft, model=dL, rho=rho, lam=lam, accepted=accept, pcg_iters=its,
                          pcg_rel_res=rel))
        if accept:
            cams, points, F = cams_t, points_t, Ft
            blk = None
            if rho > opts.rho_good:
                lam = max(lam / opts.up, opts.lambda_min)
            elif rho < opts.rho_bad:
                lam = min(lam / opts.down, opts.lambda_max)
        else:
            lam = min(lam / opts.down, opts.lambda_max)
    return cams, points, trace
