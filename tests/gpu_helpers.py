"""Shared helpers for the GPU parity tests (the oracle is imported here, in
test code only)."""
import numpy as np
import torch

import oracle as orc
import paper_2409_12190_gb300 as ba
import scenegen


def problem(sc, pix, precision="f64", **opts):
    o = ba.Options(precision=precision, huber_delta=sc.huber_delta, **opts)
    return ba.Problem(sc.cams_init, sc.points_init, sc.cam_idx, sc.pt_idx, pix, o, device="cuda")


def np64(t):
    return t.detach().to("cpu", torch.float64).numpy()


def rel_err(a, b, scale=None):
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    s = np.max(np.abs(b)) if scale is None else scale
    return float(np.max(np.abs(a - b)) / max(s, 1e-300))


def oracle_pixels_chunked(sc, chunk=1 << 20):
    out = np.empty((sc.O, 2))
    for a in range(0, sc.O, chunk):
        b = min(sc.O, a + chunk)
        out[a:b] = orc.project(sc.cams_gt, sc.points_gt, sc.cam_idx[a:b], sc.pt_idx[a:b])
    return out + sc.noise


def small_ring(C=250, P=3000, seed=2, huber=True):
    return scenegen.ring_scene(C, P, seed=seed, view_p=1.0 / 7.0,
                               outlier_frac=0.02 if huber else 0.0, outlier_px=20.0,
                               huber_delta=1.0 if huber else 0.0, name="ring-small")
