"""Seeded synthetic bundle-adjustment scenes.

This module draws every random number a scene needs and nothing else: the
ground-truth cameras and points, which camera sees which point, the pixel
noise (with outliers) and the perturbation of the initial estimate.  It holds
none of the solver's arithmetic -- in particular it never projects a point.
A caller turns a scene into observed pixels as

    pixels = projection(cams_gt, points_gt)[obs] + noise

with its own projection: the tests use the FP64 oracle, the benchmark uses the
library's projection entry point.  Both sides of a parity test therefore read
the same arrays.

Camera layout (the BAL convention used by the paper's benchmark data, Sec. V):
a camera is 9 numbers (omega[3] angle-axis, t[3], f, k1, k2); a point is
X_cam = R(omega) X + t and the camera looks down its -z axis.

Scene shapes follow the paper's workloads (Tables I-II: a few hundred to a few
thousand cameras, 3.5-8 views per point).  ``ring`` scenes put the cameras on a
circle of radius 5 around a cloud of points in [-1,1]^3, every camera facing
the centre, and let each point be seen by a contiguous window of cameras along
the ring (the banded co-visibility of a video sequence).
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np

__all__ = ["Scene", "ring_scene", "arc_scene", "batch_scenes", "config_scene",
           "subsample_points", "PoseGraph", "sphere_graph", "garage_graph", "pose_graph_config", "relabel",
           "relabel_perm"]


@dataclasses.dataclass
class Scene:
    """A seeded scene.  All float arrays are float64, index arrays int32."""
    cams_gt: np.ndarray      # [C, 9]
    points_gt: np.ndarray    # [P, 3]
    cam_idx: np.ndarray      # [O] camera of observation k
    pt_idx: np.ndarray       # [O] point of observation k
    noise: np.ndarray        # [O, 2] pixel noise (Gaussian + outliers)
    cams_init: np.ndarray    # [C, 9] perturbed initial estimate
    points_init: np.ndarray  # [P, 3]
    huber_delta: float = 0.0  # 0 = plain squared loss
    name: str = ""

    @property
    def C(self) -> int:
        return int(self.cams_gt.shape[0])

    @property
    def P(self) -> int:
        return int(self.points_gt.shape[0])

    @property
    def O(self) -> int:
        return int(self.cam_idx.shape[0])


def _finish(rng, cams_gt, points_gt, cam_idx, pt_idx, *, noise_px,
            outlier_frac, outlier_px, rot_perturb, t_perturb, pt_perturb,
            huber_delta, name, shuffle=True):
    O = cam_idx.shape[0]
    if shuffle and O > 1:
        order = rng.permutation(O)
        cam_idx = cam_idx[order]
        pt_idx = pt_idx[order]
    noise = rng.normal(0.0, noise_px, size=(O, 2))
    if outlier_frac > 0.0:
        is_out = rng.random(O) < outlier_frac
        psi = rng.uniform(0.0, 2.0 * math.pi, size=O)
        noise[is_out, 0] += outlier_px * np.cos(psi[is_out])
        noise[is_out, 1] += outlier_px * np.sin(psi[is_out])
    cams_init = cams_gt.copy()
    cams_init[:, 0:3] += rng.normal(0.0, rot_perturb, size=(cams_gt.shape[0], 3))
    cams_init[:, 3:6] += rng.normal(0.0, t_perturb, size=(cams_gt.shape[0], 3))
    points_init = points_gt + rng.normal(0.0, pt_perturb, size=points_gt.shape)
    return Scene(cams_gt=cams_gt, points_gt=points_gt,
                 cam_idx=np.ascontiguousarray(cam_idx, dtype=np.int32),
                 pt_idx=np.ascontiguousarray(pt_idx, dtype=np.int32),
                 noise=noise, cams_init=cams_init, points_init=points_init,
                 huber_delta=huber_delta, name=name)


def _windows(rng, C, counts):
    """Each point j sees cameras (s_j + m) mod C, m < counts[j]."""
    P = counts.shape[0]
    start = rng.integers(0, C, size=P)
    pt_idx = np.repeat(np.arange(P, dtype=np.int64), counts)
    first = np.repeat(np.cumsum(counts) - counts, counts)
    m = np.arange(pt_idx.shape[0], dtype=np.int64) - first
    cam_idx = (np.repeat(start, counts) + m) % C
    return cam_idx, pt_idx


def ring_scene(C: int, P: int, *, seed: int, view_p: float = 1.0 / 7.0,
               noise_px: float = 1.0, outlier_frac: float = 0.0,
               outlier_px: float = 20.0, huber_delta: float = 0.0,
               f: float = 500.0, k_std: float = 1e-3, radius: float = 5.0,
               jitter: float = 0.02, rot_perturb: float = 0.02,
               t_perturb: float = 0.05, pt_perturb: float = 0.05,
               name: str = "ring") -> Scene:
    """Cameras on a full ring facing the origin, points uniform in [-1,1]^3.

    Views per point: 2 + Geom0(view_p) (failures before the first success,
    mean 2 + (1-view_p)/view_p), capped at C; each point is seen by a
    contiguous window of cameras along the ring from a uniform start.

    The camera at ring angle phi has omega = (0, -phi, 0) (a rotation about the
    vertical axis that turns its -z axis towards the origin) plus N(0, jitter^2)
    per component, and t = (0, 0, -radius): its centre stays on the sphere of
    that radius and its optical axis passes through the origin.
    """
    rng = np.random.default_rng(seed)
    phi = 2.0 * math.pi * np.arange(C) / C
    phi = np.where(phi > math.pi, phi - 2.0 * math.pi, phi)
    cams = np.zeros((C, 9))
    cams[:, 1] = -phi
    cams[:, 0:3] += rng.normal(0.0, jitter, size=(C, 3))
    cams[:, 5] = -radius
    cams[:, 6] = f
    cams[:, 7:9] = rng.normal(0.0, k_std, size=(C, 2))
    points = rng.uniform(-1.0, 1.0, size=(P, 3))
    counts = 2 + (rng.geometric(view_p, size=P) - 1)
    counts = np.minimum(counts, C).astype(np.int64)
    cam_idx, pt_idx = _windows(rng, C, counts)
    return _finish(rng, cams, points, cam_idx, pt_idx, noise_px=noise_px,
                   outlier_frac=outlier_frac, outlier_px=outlier_px,
                   rot_perturb=rot_perturb, t_perturb=t_perturb,
                   pt_perturb=pt_perturb, huber_delta=huber_delta, name=name)


def arc_scene(C: int, P: int, *, seed: int, views_lo: int = 4,
              views_hi: int = 12, arc: float = 0.3, noise_px: float = 1.0,
              f: float = 500.0, k_std: float = 1e-3, t_std: float = 1.0,
              depth: float = 5.0, jitter: float = 0.02,
              rot_perturb: float = 0.02, t_perturb: float = 0.05,
              pt_perturb: float = 0.05, huber_delta: float = 0.0,
              name: str = "arc") -> Scene:
    """A short arc of cameras in front of a point cloud (small scenes).

    omega_i = (0, phi_i, 0) + N(0, jitter^2), phi_i evenly spaced on
    [-arc, arc]; t_i = (N(0,t_std), N(0,t_std), -depth); points uniform in
    [-1,1]^3; every point is seen by a uniform number of cameras in
    [views_lo, min(views_hi, C)], drawn uniformly without replacement.
    """
    rng = np.random.default_rng(seed)
    cams = np.zeros((C, 9))
    cams[:, 1] = np.linspace(-arc, arc, C) if C > 1 else 0.0
    cams[:, 0:3] += rng.normal(0.0, jitter, size=(C, 3))
    cams[:, 3:5] = rng.normal(0.0, t_std, size=(C, 2))
    cams[:, 5] = -depth
    cams[:, 6] = f
    cams[:, 7:9] = rng.normal(0.0, k_std, size=(C, 2))
    points = rng.uniform(-1.0, 1.0, size=(P, 3))
    hi = min(views_hi, C)
    lo = min(views_lo, hi)
    counts = rng.integers(lo, hi + 1, size=P)
    # a uniform subset without replacement: the first counts[j] entries of a
    # uniformly random permutation of the cameras
    perm = np.argsort(rng.random((P, C)), axis=1)
    take = np.arange(C)[None, :] < counts[:, None]
    chosen = np.sort(np.where(take, perm, C), axis=1)
    cam_idx = chosen[chosen < C]          # row-major: point by point
    pt_idx = np.repeat(np.arange(P), counts)
    return _finish(rng, cams, points, cam_idx, pt_idx, noise_px=noise_px,
                   outlier_frac=0.0, outlier_px=0.0, rot_perturb=rot_perturb,
                   t_perturb=t_perturb, pt_perturb=pt_perturb,
                   huber_delta=huber_delta, name=name)


def batch_scenes(n: int, *, seed: int, c_lo: int = 5, c_hi: int = 20,
                 p_lo: float = 200.0, p_hi: float = 3000.0,
                 views_lo: int = 4, views_hi: int = 10) -> list:
    """Independent sliding-window problems of uneven size.

    C_b ~ U{c_lo..c_hi}; P_b = round(exp(U[ln p_lo, ln p_hi])); views per
    point ~ U{views_lo..min(views_hi, C_b)}; each problem is an ``arc_scene``
    with its own seed derived from ``seed``.
    """
    rng = np.random.default_rng(seed)
    out = []
    for b in range(n):
        C = int(rng.integers(c_lo, c_hi + 1))
        P = int(round(math.exp(rng.uniform(math.log(p_lo), math.log(p_hi)))))
        s = int(rng.integers(0, 2**31 - 1))
        out.append(arc_scene(C, P, seed=s, views_lo=views_lo,
                             views_hi=views_hi, name=f"window{b}"))
    return out


def subsample_points(scene: Scene, n_points: int, *, seed: int = 0) -> Scene:
    """Keep ``n_points`` points (uniformly drawn) and all their observations.

    Used to time the CPU oracle on a bounded sample of a large scene.
    """
    rng = np.random.default_rng(seed)
    keep = np.sort(rng.choice(scene.P, size=min(n_points, scene.P), replace=False))
    new_id = np.full(scene.P, -1, np.int64)
    new_id[keep] = np.arange(keep.shape[0])
    sel = new_id[scene.pt_idx] >= 0
    return Scene(cams_gt=scene.cams_gt, points_gt=scene.points_gt[keep],
                 cam_idx=scene.cam_idx[sel].astype(np.int32),
                 pt_idx=new_id[scene.pt_idx[sel]].astype(np.int32),
                 noise=scene.noise[sel], cams_init=scene.cams_init,
                 points_init=scene.points_init[keep],
                 huber_delta=scene.huber_delta, name=scene.name + "-sample")


def config_scene(which: str, *, small: bool = False) -> Scene:
    """The named workloads.

    ``ba16``    16 cameras, 1,000 points, ~8k observations (4-12 views,
                uniform), 1 px noise, seed 1.
    ``ba250``   250 cameras, 60,000 points, ~480k observations (2+Geom0(1/7)
                views), 1 px noise + 2 % outliers at 20 px, Huber delta 1 px,
                seed 2.
    ``ba4000``  4,000 cameras, 1.2M points, ~8M observations (2+Geom0(1/5.7)
                views), 1 px noise, seed 3.
    ``ba64``    64 cameras, 10,000 points, ~80k observations, seed 5.
    ``small=True`` shrinks the point count (same cameras and recipe) for the
    parity tests that must run the oracle in seconds.
    """
    if which == "ba16":
        return arc_scene(16, 1000, seed=1, name="ba16")
    if which == "ba250":
        return ring_scene(250, 6000 if small else 60000, seed=2,
                          view_p=1.0 / 7.0, outlier_frac=0.02, outlier_px=20.0,
                          huber_delta=1.0, name="ba250")
    if which == "ba4000":
        return ring_scene(4000, 12000 if small else 1200000, seed=3,
                          view_p=1.0 / 5.7, name="ba4000")
    if which == "ba64":
        return ring_scene(64, 1000 if small else 10000, seed=5,
                          view_p=1.0 / 7.0, name="ba64")
    raise ValueError(f"unknown scene {which!r}")


# --------------------------------------------------------------------------
# Pose graphs (the paper's PGO problem, Sec. IV-D)
# --------------------------------------------------------------------------

@dataclasses.dataclass
class PoseGraph:
    """A seeded pose graph.  A caller builds the measured relative poses and
    the initial estimate with its own SE(3) arithmetic as

        T_ij   = Exp(noise_e) zeta_i^{-1} zeta_j      (left noise: at the
                                                        truth r_e = -noise_e)
        zeta_i(init) = Exp(drift_i) zeta_i

    Tangent vectors are (translation, rotation); poses are (t, q) with the
    quaternion (qx, qy, qz, qw); info is the upper triangle of each edge's
    6 x 6 information matrix, row by row, matched to the noise's covariance."""
    poses_gt: np.ndarray   # [N, 7]
    ei: np.ndarray         # [E] int32
    ej: np.ndarray         # [E] int32
    noise: np.ndarray      # [E, 6]
    info: np.ndarray       # [E, 21]
    drift: np.ndarray      # [N, 6]
    name: str = ""

    @property
    def N(self) -> int:
        return int(self.poses_gt.shape[0])

    @property
    def E(self) -> int:
        return int(self.ei.shape[0])


def _yaw_pitch_quat(yaw, pitch):
    """Unit quaternion (x, y, z, w) of Rz(yaw) Ry(pitch)."""
    sz, cz = np.sin(0.5 * yaw), np.cos(0.5 * yaw)
    sy, cy = np.sin(0.5 * pitch), np.cos(0.5 * pitch)
    return np.stack([-sz * sy, cz * sy, sz * cy, cz * cy], -1)


def _graph_noise(rng, E, sigma_t, sigma_r, full_info):
    """Edge noise and the matching information matrices: covariance
    Q diag(s^2) Q^T with s = (sigma_t x 3, sigma_r x 3) and Q = I, or a random
    orthogonal Q (full_info); info = its inverse."""
    s = np.array([sigma_t] * 3 + [sigma_r] * 3)
    z = rng.normal(size=(E, 6)) * s
    iu = np.triu_indices(6)
    if not full_info:
        info = np.zeros((E, 21))
        info[:, [k for k, (a, b) in enumerate(zip(*iu)) if a == b]] = 1.0 / (s * s)
        return z, info
    Q, _ = np.linalg.qr(rng.normal(size=(E, 6, 6)))
    noise = np.einsum("eab,eb->ea", Q, z)
    Om = np.einsum("eab,b,ecb->eac", Q, 1.0 / (s * s), Q)
    return noise, Om[:, iu[0], iu[1]]


def _pick(rng, cand, n):
    cand = np.asarray(cand, dtype=np.int64).reshape(-1, 2)
    if n is not None and n < len(cand):
        cand = cand[np.sort(rng.choice(len(cand), size=n, replace=False))]
    return cand


def _graph(rng, pos, quat, closures, *, sigma_t, sigma_r, drift_t, drift_r, full_info, name):
    N = pos.shape[0]
    odo = np.stack([np.arange(N - 1), np.arange(1, N)], 1)
    edges = np.concatenate([odo, closures], 0)
    noise, info = _graph_noise(rng, len(edges), sigma_t, sigma_r, full_info)
    # initial estimate: a random walk along the node order (odometry drift),
    # node 0 exact
    steps = rng.normal(size=(N, 6)) * np.array([drift_t] * 3 + [drift_r] * 3)
    steps[0] = 0.0
    return PoseGraph(poses_gt=np.concatenate([pos, quat], 1), ei=edges[:, 0].astype(np.int32),
                     ej=edges[:, 1].astype(np.int32), noise=noise, info=info, drift=np.cumsum(steps, 0),
                     name=name)


def sphere_graph(rings: int, per_ring: int, *, seed: int, n_closures=None, radius: float = 50.0,
                 sigma_t: float = 0.05, sigma_r: float = 0.01, drift_t: float = 0.02,
                 drift_r: float = 0.004, full_info: bool = False, name: str = "sphere") -> PoseGraph:
    """Poses on a sphere, visited ring by ring (latitude rings of per_ring
    nodes, heading along the ring): odometry edges between consecutive nodes
    and loop closures from node (ring r, index m) to ring r+1 at indices
    m-1, m, m+1 (a random n_closures of them)."""
    rng = np.random.default_rng(seed)
    k = np.arange(rings * per_ring)
    ring, m = k // per_ring, k % per_ring
    lat = -0.5 * np.pi + np.pi * (ring + 0.5) / rings
    lon = 2.0 * np.pi * m / per_ring
    pos = radius * np.stack([np.cos(lat) * np.cos(lon), np.cos(lat) * np.sin(lon), np.sin(lat)], 1)
    quat = _yaw_pitch_quat(lon + 0.5 * np.pi, -lat)
    cand = [(r * per_ring + a, (r + 1) * per_ring + (a + d) % per_ring)
            for r in range(rings - 1) for a in range(per_ring) for d in (-1, 0, 1)]
    return _graph(rng, pos, quat, _pick(rng, cand, n_closures), sigma_t=sigma_t, sigma_r=sigma_r,
                  drift_t=drift_t, drift_r=drift_r, full_info=full_info, name=name)


def garage_graph(laps: int, per_lap: int, *, seed: int, n_closures=None, side: float = 40.0,
                 rise: float = 3.0, sigma_t: float = 0.02, sigma_r: float = 0.005, drift_t: float = 0.01,
                 drift_r: float = 0.002, full_info: bool = False, name: str = "garage") -> PoseGraph:
    """A drive round a square ramp (a parking garage): per_lap nodes per lap,
    rising by `rise` per lap, heading along the path; odometry edges and loop
    closures from each node to the previous lap's nodes at offsets -2..2 (a
    random n_closures of them)."""
    rng = np.random.default_rng(seed)
    k = np.arange(laps * per_lap)
    s = 4.0 * (k % per_lap) / per_lap            # position along the square, 0..4
    side_i = np.floor(s).astype(int)
    f = s - side_i
    corners = side * np.array([[0.0, 0.0], [1.0, 0.0], [1.0, 1.0], [0.0, 1.0], [0.0, 0.0]])
    xy = corners[side_i] + f[:, None] * (corners[side_i + 1] - corners[side_i])
    z = rise * k / per_lap
    pos = np.concatenate([xy, z[:, None]], 1)
    yaw = 0.5 * np.pi * side_i
    pitch = -np.arctan2(rise, 4.0 * side) * np.ones_like(yaw)
    quat = _yaw_pitch_quat(yaw, pitch)
    cand = [(a - per_lap + d, a) for a in range(per_lap, laps * per_lap) for d in (-2, -1, 0, 1, 2)
            if 0 <= a - per_lap + d < a - 1]
    return _graph(rng, pos, quat, _pick(rng, cand, n_closures), sigma_t=sigma_t, sigma_r=sigma_r,
                  drift_t=drift_t, drift_r=drift_r, full_info=full_info, name=name)


def relabel_perm(N: int, *, seed: int) -> np.ndarray:
    """The seeded random renumbering of relabel: node n becomes perm[n]."""
    return np.random.default_rng(seed).permutation(N)


def relabel(graph: PoseGraph, *, seed: int) -> PoseGraph:
    """The same graph with its nodes renumbered by a seeded random
    permutation (node n becomes relabel_perm(N, seed)[n]; edges, noise and
    information keep their order)."""
    perm = relabel_perm(graph.N, seed=seed)
    inv = np.empty_like(perm)
    inv[perm] = np.arange(graph.N)
    return PoseGraph(poses_gt=graph.poses_gt[inv], ei=perm[graph.ei].astype(np.int32),
                     ej=perm[graph.ej].astype(np.int32), noise=graph.noise.copy(), info=graph.info.copy(),
                     drift=graph.drift[inv], name=graph.name + "-relabelled")


def pose_graph_config(which: str) -> PoseGraph:
    """The named pose graphs (node and edge counts of the paper's PGO
    benchmark files, Table VIII; synthetic geometry and noise).

    ``sphere2500``  2,500 nodes (50 rings of 50), 9,799 edges, seed 21.
    ``garage1661``  1,661 nodes (11 laps of 151), 6,275 edges, seed 22.
    ``sphere100``   100 nodes (10 rings of 10), full information matrices,
                    seed 23: the small case the oracle runs in seconds.
    """
    if which == "sphere2500":
        return sphere_graph(50, 50, seed=21, n_closures=9799 - 2499, name="sphere2500")
    if which == "garage1661":
        return garage_graph(11, 151, seed=22, n_closures=6275 - 1660, name="garage1661")
    if which == "sphere100":
        return sphere_graph(10, 10, seed=23, radius=10.0, full_info=True, name="sphere100")
    raise ValueError(f"unknown pose graph {which!r}")
