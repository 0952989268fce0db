"""Pose-graph optimisation on the GPU (Sec. IV-D, Eqs. 3-4) against the
oracle: residuals, Jacobians, normal-equation blocks, the damped product,
the PCG and Cholesky solves, the LM trace, and the full-size graphs
(sphere2500, garage1661) element by element at the initial poses and by the
oracle's cost and gradient at the GPU's converged poses."""
import numpy as np
import pytest
import torch

import paper_2409_12190_gb300 as ba
import scenegen
from oracle import LMOptions
from oracle import pgo
from paper_2409_12190_gb300.pgo import PoseGraph, synthesize

pytestmark = pytest.mark.gpu


def _inputs(g):
    Ts, Tms, infos, Tg = pgo.graph_inputs(g)
    return Ts, Tms, infos, Tg, pgo.matrices_to_poses(Ts), pgo.matrices_to_poses(Tms)


def _graph(full_info=True, seed=3, noise=True):
    g = scenegen.sphere_graph(4, 6, seed=seed, radius=5.0, full_info=full_info, name="tiny")
    if not noise:
        g.noise[:] = 0.0
    return g


def _make(g, P7, M7, fixed=(0,), **opts):
    return PoseGraph(P7, g.ei, g.ej, M7, g.info, fixed=fixed, options=ba.Options(**opts))


def _mask(N, fixed):
    m = np.zeros(N, bool)
    m[list(fixed)] = True
    return m


def _rel(a, b):
    a, b = np.asarray(a, np.float64), np.asarray(b, np.float64)
    return float(np.max(np.abs(a - b)) / max(np.max(np.abs(b)), 1e-300))


def _upper(M):
    iu = np.triu_indices(6)
    return M[:, iu[0], iu[1]]


def test_synthesize_matches_the_oracle():
    g = scenegen.pose_graph_config("sphere100")
    _, Tms, _, _ = pgo.graph_inputs(g)
    meas, init = synthesize(g.poses_gt, g.ei, g.ej, g.noise, g.drift)
    Tm_gpu = pgo.poses_to_matrices(meas.cpu().numpy())
    Ts, _, _, _ = pgo.graph_inputs(g)
    assert np.max(np.abs(Tm_gpu - Tms)) < 1e-12
    assert np.max(np.abs(pgo.poses_to_matrices(init.cpu().numpy()) - Ts)) < 1e-12


@pytest.mark.parametrize("full_info", [True, False])
def test_linearize_matches_the_oracle(full_info):
    g = _graph(full_info=full_info)
    Ts, Tms, infos, _, P7, M7 = _inputs(g)
    blk = pgo.assemble(Ts, g.ei, g.ej, Tms, infos)
    with _make(g, P7, M7) as pg:
        out = pg.linearize()
    assert _rel(out["r"].cpu(), blk["r"]) < 1e-12
    assert _rel(out["A"].cpu(), blk["A"]) < 1e-12
    assert _rel(out["B"].cpu(), blk["B"]) < 1e-12
    assert _rel(out["Hd"].cpu(), _upper(blk["Hd"])) < 1e-12
    assert _rel(out["g"].cpu(), blk["g"]) < 1e-12
    F = pgo.cost(Ts, g.ei, g.ej, Tms, infos)
    assert abs(out["cost"] - F) <= 1e-12 * F


def test_large_rotation_residuals_match_the_oracle():
    """Residual rotations up to ~3 rad (the log near pi) and tiny ones."""
    rng = np.random.default_rng(11)
    N, E = 12, 30
    P7 = np.concatenate([rng.normal(size=(N, 3)) * 3, rng.normal(size=(N, 4))], 1)
    ei = rng.integers(0, N, E).astype(np.int32)
    ej = ((ei + rng.integers(1, N, E)) % N).astype(np.int32)
    Ts = pgo.poses_to_matrices(P7)
    Tms = []
    for k, (i, j) in enumerate(zip(ei, ej)):
        phi = rng.normal(size=3)
        ang = [3.1, 2.0, 1e-7, 1e-3, 0.05, 0.5][k % 6]
        xi = np.concatenate([rng.normal(size=3), phi / np.linalg.norm(phi) * ang])
        # residual Log(Ti^-1 Tj Tm^-1) with Tm = Exp(-xi) Ti^-1 Tj is xi
        Tms.append(pgo.se3_exp(-xi) @ pgo.se3_inv(Ts[i]) @ Ts[j])
    Tms = np.stack(Tms)
    info = np.tile(pgo.info_upper(np.eye(6)), (E, 1))
    gg = scenegen.PoseGraph(poses_gt=P7, ei=ei, ej=ej, noise=np.zeros((E, 6)), info=info, drift=np.zeros((N, 6)))
    blk = pgo.assemble(Ts, ei, ej, Tms, np.tile(np.eye(6), (E, 1, 1)))
    with _make(gg, P7, pgo.matrices_to_poses(Tms), fixed=()) as pg:
        out = pg.linearize()
    assert np.max(np.abs(out["r"].cpu().numpy() - blk["r"])) < 1e-11
    assert _rel(out["A"].cpu(), blk["A"]) < 1e-10


def test_damped_product_matches_the_oracle():
    g = _graph()
    Ts, Tms, infos, _, P7, M7 = _inputs(g)
    blk = pgo.assemble(Ts, g.ei, g.ej, Tms, infos)
    fixed = (0, 7)
    m = _mask(g.N, fixed)
    x = np.random.default_rng(2).normal(size=(g.N, 6))
    D = pgo.damping(blk, 1e-3, LMOptions())
    xm = x * ~m[:, None]
    want = (pgo.matvec(blk, xm) + D * xm) * ~m[:, None]
    with _make(g, P7, M7, fixed=fixed) as pg:
        y = pg.matvec(1e-3, torch.tensor(x)).cpu().numpy()
    assert _rel(y, want) < 1e-12


@pytest.mark.parametrize("k", [1, 5, 20])
def test_pcg_iterates_match_the_oracle(k):
    """k PCG iterations from the same start: the same iteration in both."""
    g = _graph()
    Ts, Tms, infos, _, P7, M7 = _inputs(g)
    blk = pgo.assemble(Ts, g.ei, g.ej, Tms, infos)
    want, its, _ = pgo.solve_damped(blk, 1e-3, LMOptions(solver="pcg", pcg_tol=0.0, pcg_maxiter=k),
                                    _mask(g.N, (0,)))
    with _make(g, P7, M7) as pg:
        dx, gits, _ = pg.damped_solve(1e-3, k, 0.0)
    assert gits == its == k
    assert _rel(dx.cpu(), want) < 1e-9


@pytest.mark.parametrize("solver", ["pcg", "cholesky"])
def test_exact_solves_match_the_oracle_cholesky(solver):
    g = _graph()
    Ts, Tms, infos, _, P7, M7 = _inputs(g)
    blk = pgo.assemble(Ts, g.ei, g.ej, Tms, infos)
    fixed = (0, 9)
    want, _, _ = pgo.solve_damped(blk, 1e-4, LMOptions(solver="cholesky"), _mask(g.N, fixed))
    with _make(g, P7, M7, fixed=fixed, solver=solver) as pg:
        dx, its, rel = pg.damped_solve(1e-4, 2000, 1e-13)
    assert _rel(dx.cpu(), want) < 1e-9
    assert np.all(dx.cpu().numpy()[list(fixed)] == 0.0)
    if solver == "pcg":
        assert rel <= 1e-13 and its > 10


def test_pcg_with_a_hub_node_matches_the_oracle():
    """A star (node 0 joined to every node) plus a chain, 700 nodes: the
    first node group's incidence slots exceed the shared-memory budget of
    the register-resident PCG, so the general kernel runs; its iterates and
    its converged solve against the oracle."""
    rng = np.random.default_rng(31)
    N = 700
    ei = np.concatenate([np.zeros(N - 1, np.int32), np.arange(1, N - 1, dtype=np.int32)])
    ej = np.concatenate([np.arange(1, N, dtype=np.int32), np.arange(2, N, dtype=np.int32)])
    E = len(ei)
    P7 = np.concatenate([rng.normal(size=(N, 3)) * 5, rng.normal(size=(N, 4))], 1)
    Ts = pgo.poses_to_matrices(P7)
    Tms = np.stack([pgo.se3_exp(rng.normal(size=6) * 0.05) @ pgo.se3_inv(Ts[i]) @ Ts[j] for i, j in zip(ei, ej)])
    info = np.tile(pgo.info_upper(np.eye(6)), (E, 1))
    gg = scenegen.PoseGraph(poses_gt=P7, ei=ei, ej=ej, noise=np.zeros((E, 6)), info=info, drift=np.zeros((N, 6)))
    blk = pgo.assemble(Ts, ei, ej, Tms, np.tile(np.eye(6), (E, 1, 1)))
    m = _mask(N, (5,))
    it_ref, _, _ = pgo.solve_damped(blk, 1e-3, LMOptions(solver="pcg", pcg_tol=0.0, pcg_maxiter=12), m)
    exact, _, _ = pgo.solve_damped(blk, 1e-3, LMOptions(solver="cholesky"), m)
    with _make(gg, P7, pgo.matrices_to_poses(Tms), fixed=(5,)) as pg:
        dx, its, _ = pg.damped_solve(1e-3, 12, 0.0)
        dx2, _, rel = pg.damped_solve(1e-3, 5000, 1e-13)
    assert its == 12 and _rel(dx.cpu(), it_ref) < 1e-9
    assert rel <= 1e-13 and _rel(dx2.cpu(), exact) < 1e-8


def test_pcg_grid_stride_on_a_large_graph_matches_the_oracle():
    """12,000 poses (a chain with closures every 50 poses): more node groups
    than the PCG grid holds resident blocks, so blocks stride over several
    groups; 10 iterations against the oracle's."""
    rng = np.random.default_rng(41)
    N = 12000
    ei = np.concatenate([np.arange(N - 1), np.arange(0, N - 50, 7)]).astype(np.int32)
    ej = np.concatenate([np.arange(1, N), np.arange(50, N, 7)]).astype(np.int32)
    E = len(ei)
    P7 = np.concatenate([rng.normal(size=(N, 3)) * 5, rng.normal(size=(N, 4))], 1)
    Ts = pgo.poses_to_matrices(P7)
    Tms = np.stack([pgo.se3_exp(rng.normal(size=6) * 0.05) @ pgo.se3_inv(Ts[i]) @ Ts[j] for i, j in zip(ei, ej)])
    info = np.tile(pgo.info_upper(np.eye(6)), (E, 1))
    gg = scenegen.PoseGraph(poses_gt=P7, ei=ei, ej=ej, noise=np.zeros((E, 6)), info=info, drift=np.zeros((N, 6)))
    blk = pgo.assemble(Ts, ei, ej, Tms, np.tile(np.eye(6), (E, 1, 1)))
    m = _mask(N, (0,))
    want, _, _ = pgo.solve_damped(blk, 1e-3, LMOptions(solver="pcg", pcg_tol=0.0, pcg_maxiter=10), m)
    with _make(gg, P7, pgo.matrices_to_poses(Tms)) as pg:
        dx, its, _ = pg.damped_solve(1e-3, 10, 0.0)
    assert its == 10 and _rel(dx.cpu(), want) < 1e-9


@pytest.mark.parametrize("kind", ["chain", "random"])
def test_banded_cholesky_matches_the_oracle(kind):
    """The Cholesky solver factors within the band of the node order: a
    chain (half-bandwidth 11 unknowns, inside one 32-wide tile) and a random
    graph (band = the whole matrix), against the oracle's dense Cholesky."""
    rng = np.random.default_rng(21 if kind == "chain" else 22)
    N = 70
    if kind == "chain":
        ei = np.arange(N - 1, dtype=np.int32)
        ej = ei + 1
    else:
        ei = rng.integers(0, N, 250).astype(np.int32)
        ej = ((ei + rng.integers(1, N, 250)) % N).astype(np.int32)
        ei = np.concatenate([ei, np.arange(N - 1, dtype=np.int32), [0]]).astype(np.int32)
        ej = np.concatenate([ej, np.arange(1, N, dtype=np.int32), [N - 1]]).astype(np.int32)
    E = len(ei)
    P7 = np.concatenate([rng.normal(size=(N, 3)) * 3, rng.normal(size=(N, 4))], 1)
    Ts = pgo.poses_to_matrices(P7)
    Tms = np.stack([pgo.se3_exp(rng.normal(size=6) * 0.1) @ pgo.se3_inv(Ts[i]) @ Ts[j] for i, j in zip(ei, ej)])
    Om = np.stack([np.diag(rng.uniform(0.5, 2.0, 6)) for _ in range(E)])
    info = np.stack([pgo.info_upper(M) for M in Om])
    gg = scenegen.PoseGraph(poses_gt=P7, ei=ei, ej=ej, noise=np.zeros((E, 6)), info=info, drift=np.zeros((N, 6)))
    blk = pgo.assemble(Ts, ei, ej, Tms, Om)
    fixed = (0, 33)
    want, _, _ = pgo.solve_damped(blk, 1e-3, LMOptions(solver="cholesky"), _mask(N, fixed))
    with _make(gg, P7, pgo.matrices_to_poses(Tms), fixed=fixed, solver="cholesky") as pg:
        dx, _, rel = pg.damped_solve(1e-3, 0, 0.0)
    assert rel == 0.0
    assert _rel(dx.cpu(), want) < 1e-9


@pytest.mark.parametrize("solver", ["cholesky", "pcg"])
def test_lm_trace_matches_the_oracle(solver):
    """sphere100, 8 trials with exact solves (Cholesky, or PCG to 1e-13):
    every trial's costs and decision at 1e-9, final poses at 1e-9."""
    g = scenegen.pose_graph_config("sphere100")
    Ts, Tms, infos, _, P7, M7 = _inputs(g)
    opts = LMOptions(solver="cholesky")
    T_ref, ref = pgo.lm(Ts, g.ei, g.ej, Tms, infos, 8, opts, _mask(g.N, (0,)))
    with _make(g, P7, M7, solver=solver, pcg_tol=1e-13, pcg_maxiter=5000) as pg:
        pg.solve(8)
        st = pg.stats()
        poses = pg.poses().cpu().numpy()
        F, _ = pg.scalars()
    assert len(st) == 8
    for t, (a, b) in enumerate(zip(st, ref)):
        assert a["accepted"] == b["accepted"], t
        for key in ("cost", "cost_trial", "model"):
            assert abs(a[key] - b[key]) <= 1e-9 * abs(b["cost"]), (t, key, a[key], b[key])
        assert a["lam"] == b["lam"], t
    assert np.max(np.abs(pgo.poses_to_matrices(poses) - T_ref)) < 1e-9 * 10.0
    assert abs(F - pgo.cost(pgo.poses_to_matrices(poses), g.ei, g.ej, Tms, infos)) <= 1e-12 * F


def test_cholesky_on_a_shuffled_numbering_matches_the_oracle():
    """sphere100 with its poses renumbered at random: the band of the node
    order is then nearly the whole matrix and the Cholesky solver factors in
    its reverse Cuthill-McKee order; the 8-trial trace against the
    oracle's (which solves in the node order)."""
    g = scenegen.relabel(scenegen.pose_graph_config("sphere100"), seed=4)
    Ts, Tms, infos, _, P7, M7 = _inputs(g)
    fixed = (int(np.argmin(np.abs(np.arange(g.N) - 50))),)
    T_ref, ref = pgo.lm(Ts, g.ei, g.ej, Tms, infos, 8, LMOptions(solver="cholesky"), _mask(g.N, fixed))
    with _make(g, P7, M7, fixed=fixed, solver="cholesky") as pg:
        pg.solve(8)
        st = pg.stats()
        poses = pg.poses().cpu().numpy()
    for t, (a, b) in enumerate(zip(st, ref)):
        assert a["accepted"] == b["accepted"], t
        for key in ("cost", "cost_trial", "model"):
            assert abs(a[key] - b[key]) <= 1e-9 * abs(b["cost"]), (t, key, a[key], b[key])
    assert np.max(np.abs(pgo.poses_to_matrices(poses) - T_ref)) < 1e-8


def test_noise_free_graph_reaches_the_truth():
    g = _graph(noise=False)
    Ts, Tms, infos, Tg, P7, M7 = _inputs(g)
    with _make(g, P7, M7, pcg_tol=1e-12, pcg_maxiter=2000) as pg:
        F0, _ = pg.scalars()
        pg.solve(12)
        F, _ = pg.scalars()
        poses = pg.poses().cpu().numpy()
    assert F0 > 1.0 and F < 1e-16 * F0
    assert np.max(np.abs(pgo.poses_to_matrices(poses) - Tg)) < 1e-7


def test_set_poses_and_fixed_poses():
    g = _graph()
    Ts, Tms, infos, _, P7, M7 = _inputs(g)
    with _make(g, P7, M7, fixed=(0, 3)) as pg:
        pg.solve(3)
        out = pg.poses().cpu().numpy()
        # held: bit for bit what the input normalised to
        assert np.allclose(out[[0, 3]], pgo.matrices_to_poses(Ts[[0, 3]]), rtol=0, atol=1e-15)
        pg.solve(2)
        assert np.array_equal(pg.poses().cpu().numpy()[[0, 3]], out[[0, 3]])
        pg.set_poses(P7)
        F, _ = pg.scalars()
        assert abs(F - pgo.cost(Ts, g.ei, g.ej, Tms, infos)) <= 1e-12 * F


@pytest.mark.parametrize("case", ["isolated", "duplicate", "two"])
def test_degenerate_graphs_match_the_oracle(case):
    """A pose with no edge (H_ii = 0: the damping's clamp keeps its block
    SPD and its step is 0), two edges between the same pair (summed in
    order), and the smallest graph (two poses, one edge)."""
    rng = np.random.default_rng(51)
    if case == "two":
        N, ei, ej = 2, np.array([0], np.int32), np.array([1], np.int32)
    else:
        N = 12
        ei = np.arange(N - 2, dtype=np.int32)
        ej = ei + 1
        if case == "duplicate":
            ei = np.concatenate([ei, [3, 3]]).astype(np.int32)
            ej = np.concatenate([ej, [7, 7]]).astype(np.int32)
        # "isolated": pose N - 1 has no edge
    E = len(ei)
    P7 = np.concatenate([rng.normal(size=(N, 3)) * 3, rng.normal(size=(N, 4))], 1)
    Ts = pgo.poses_to_matrices(P7)
    Tms = np.stack([pgo.se3_exp(rng.normal(size=6) * 0.2) @ pgo.se3_inv(Ts[i]) @ Ts[j] for i, j in zip(ei, ej)])
    Om = np.stack([np.diag(rng.uniform(0.5, 2.0, 6)) for _ in range(E)])
    info = np.stack([pgo.info_upper(M) for M in Om])
    gg = scenegen.PoseGraph(poses_gt=P7, ei=ei, ej=ej, noise=np.zeros((E, 6)), info=info, drift=np.zeros((N, 6)))
    # two poses and one edge: the cost reaches 0 exactly after the second
    # trial, where further decisions compare rounding noise
    iters = 2 if case == "two" else 6
    T_ref, ref = pgo.lm(Ts, ei, ej, Tms, Om, iters, LMOptions(solver="cholesky"), _mask(N, (0,)))
    F0 = ref[0]["cost"]
    for solver in ("cholesky", "pcg"):
        with _make(gg, P7, pgo.matrices_to_poses(Tms), solver=solver, pcg_tol=1e-13, pcg_maxiter=500) as pg:
            pg.solve(iters)
            st = pg.stats()
            poses = pgo.poses_to_matrices(pg.poses().cpu().numpy())
        assert len(st) == iters
        for t, (a, b) in enumerate(zip(st, ref)):
            assert a["accepted"] == b["accepted"], (solver, t)
            assert abs(a["cost_trial"] - b["cost_trial"]) <= 1e-9 * b["cost"] + 1e-15 * F0, (solver, t, a, b)
        assert np.max(np.abs(poses - T_ref)) < 1e-8, solver
        if case == "isolated":
            assert np.max(np.abs(poses[N - 1] - Ts[N - 1])) < 1e-14


def test_c_program_solves_a_pose_graph(tmp_path):
    """A C99 program solves sphere100 through include/ba.h with host
    pointers only; its per-trial costs and final poses match the oracle's LM
    with the Cholesky solve."""
    import os
    import shutil
    import subprocess
    if shutil.which("gcc") is None:
        pytest.skip("no C compiler")
    from paper_2409_12190_gb300 import build as b
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    libdir = os.path.dirname(b.build())
    exe = tmp_path / "pgo_from_c"
    subprocess.run(["gcc", "-std=c99", "-Wall", "-Wextra", "-Werror", "-I", os.path.join(root, "include"),
                    os.path.join(root, "tests", "c", "pgo_from_c.c"), "-L", libdir, "-lba_gb300",
                    f"-Wl,-rpath,{libdir}", "-o", str(exe)], check=True)
    g = scenegen.pose_graph_config("sphere100")
    Ts, Tms, infos, _, P7, M7 = _inputs(g)
    iters = 8
    fixed = np.zeros(g.N, np.uint8)
    fixed[0] = 1
    path = tmp_path / "graph.bin"
    with open(path, "wb") as f:
        np.array([g.N, g.E, iters, 1, 0], dtype=np.int32).tofile(f)  # solver 1: Cholesky
        np.array([0.0], dtype=np.float64).tofile(f)
        np.ascontiguousarray(P7, dtype=np.float64).tofile(f)
        np.ascontiguousarray(g.ei, dtype=np.int32).tofile(f)
        np.ascontiguousarray(g.ej, dtype=np.int32).tofile(f)
        np.ascontiguousarray(M7, dtype=np.float64).tofile(f)
        np.ascontiguousarray(g.info, dtype=np.float64).tofile(f)
        fixed.tofile(f)
    out = subprocess.run([str(exe), str(path)], capture_output=True, text=True, timeout=300)
    assert out.returncode == 0, out.stderr
    lines = out.stdout.split("\n")
    trials = [ln.split() for ln in lines if ln.startswith("trial ")]
    poses = np.array([float(ln.split()[1]) for ln in lines if ln.startswith("pose ")]).reshape(g.N, 7)
    T_ref, ref = pgo.lm(Ts, g.ei, g.ej, Tms, infos, iters, LMOptions(solver="cholesky"), _mask(g.N, (0,)))
    assert len(trials) == iters
    for t, r in zip(trials, ref):
        assert abs(float(t[2]) - r["cost"]) <= 1e-9 * r["cost"], (t, r)
        assert abs(float(t[3]) - r["cost_trial"]) <= 1e-9 * r["cost"], (t, r)
        assert bool(int(t[4])) == r["accepted"], (t, r)
    assert np.max(np.abs(pgo.poses_to_matrices(poses) - T_ref)) < 1e-8


def test_invalid_inputs_are_reported():
    g = _graph()
    _, _, _, _, P7, M7 = _inputs(g)
    bad = g.ej.copy()
    bad[3] = g.N
    with pytest.raises(ba.BAError, match="INVALID_ARG"):
        PoseGraph(P7, g.ei, bad, M7, g.info)
    bad = g.ej.copy()
    bad[2] = g.ei[2]
    with pytest.raises(ba.BAError, match="INVALID_ARG"):
        PoseGraph(P7, g.ei, bad, M7, g.info)
    P = P7.copy()
    P[1, 0] = np.nan
    with pytest.raises(ba.BAError, match="NONFINITE"):
        PoseGraph(P, g.ei, g.ej, M7, g.info)
    P = P7.copy()
    P[1, 3:] = 0.0
    with pytest.raises(ba.BAError, match="NONFINITE"):
        PoseGraph(P, g.ei, g.ej, M7, g.info)
    with pytest.raises(ba.BAError, match="INVALID_ARG"):
        PoseGraph(P7, g.ei, g.ej, M7, g.info, options=ba.Options(huber_delta=1.0))
    with pytest.raises(ValueError):
        PoseGraph(P7, g.ei, g.ej, M7, g.info, options=ba.Options(precision="f32"))


def test_banded_cholesky_on_a_graph_larger_than_a_dense_factorisation_takes():
    """A 62 x 50 sphere (3,100 poses, 18,600 unknowns, more than
    BA_DENSE_MAX_DIM): only the band tiles are stored.  One damped solve
    with pose 0 fixed: (H + D) dx = -g to 1e-10 over the free poses, and dx
    against PCG run to 1e-12 on the same graph."""
    big = scenegen.sphere_graph(62, 50, seed=1, name="big")
    _, _, _, _, P7, M7 = _inputs(big)
    lam = 1e-3
    with _make(big, P7, M7, solver="cholesky") as pc:
        dx, its, rel = pc.damped_solve(lam, 0, 0.0)
        g = pc.linearize()["g"]
        y = pc.matvec(lam, dx)
    with _make(big, P7, M7, pcg_tol=1e-12, pcg_maxiter=20000) as pp:
        dx_p, _, rel_p = pp.damped_solve(lam, 20000, 1e-12)
    assert its == 0 and rel == 0.0 and rel_p <= 1e-12
    res = (y + g)[1:].cpu().numpy()
    assert np.max(np.abs(res)) <= 1e-10 * float(g[1:].abs().max())
    assert np.all(dx[0].cpu().numpy() == 0.0)
    assert _rel(dx.cpu(), dx_p.cpu()) < 1e-6


# --------------------------------------------------------------------------
# Full size: the paper's benchmark graph sizes (synthetic)
# --------------------------------------------------------------------------

@pytest.mark.parametrize("which", ["sphere2500", "garage1661"])
def test_full_size_blocks_and_product_match_the_oracle(which):
    g = scenegen.pose_graph_config(which)
    Ts, Tms, infos, _, P7, M7 = _inputs(g)
    blk = pgo.assemble(Ts, g.ei, g.ej, Tms, infos)
    with _make(g, P7, M7) as pg:
        out = pg.linearize()
        x = np.random.default_rng(4).normal(size=(g.N, 6))
        y = pg.matvec(1e-4, torch.tensor(x)).cpu().numpy()
        dx, its, _ = pg.damped_solve(1e-4, 10, 0.0)
    assert _rel(out["r"].cpu(), blk["r"]) < 1e-11
    assert _rel(out["B"].cpu(), blk["B"]) < 1e-11
    assert _rel(out["g"].cpu(), blk["g"]) < 1e-11
    F = pgo.cost(Ts, g.ei, g.ej, Tms, infos)
    assert abs(out["cost"] - F) <= 1e-11 * F
    m = _mask(g.N, (0,))
    xm = x * ~m[:, None]
    D = pgo.damping(blk, 1e-4, LMOptions())
    assert _rel(y, (pgo.matvec(blk, xm) + D * xm) * ~m[:, None]) < 1e-11
    want, wits, _ = pgo.solve_damped(blk, 1e-4, LMOptions(solver="pcg", pcg_tol=0.0, pcg_maxiter=10), m)
    assert its == wits == 10
    assert _rel(dx.cpu(), want) < 1e-9


@pytest.mark.parametrize("which,solver", [("sphere2500", "pcg"), ("garage1661", "pcg"), ("sphere2500", "cholesky"),
                                          ("garage1661", "cholesky")])
def test_full_size_lm_converges_to_a_stationary_point(which, solver):
    """The bench configuration run to convergence with either solver (the
    banded Cholesky factors garage1661 in its reverse Cuthill-McKee order):
    the GPU's reported cost equals the oracle's cost at the GPU's poses
    (1e-9), every accepted trial lowered it, and the oracle's gradient there
    has fallen by 1e-4 of the starting gradient (a stationarity certificate
    independent of the GPU's own arithmetic)."""
    g = scenegen.pose_graph_config(which)
    Ts, Tms, infos, _, P7, M7 = _inputs(g)
    with _make(g, P7, M7, solver=solver, pcg_tol=1e-6, pcg_maxiter=5000) as pg:
        pg.solve(30)
        st = pg.stats()
        F, _ = pg.scalars()
        poses = pg.poses().cpu().numpy()
    T = pgo.poses_to_matrices(poses)
    Fo = pgo.cost(T, g.ei, g.ej, Tms, infos)
    assert abs(F - Fo) <= 1e-9 * Fo
    costs = [s["cost"] for s in st]
    assert all(b <= a for a, b in zip(costs, costs[1:]))
    g0 = pgo.assemble(Ts, g.ei, g.ej, Tms, infos)["g"][1:]
    g1 = pgo.assemble(T, g.ei, g.ej, Tms, infos)["g"][1:]
    assert np.linalg.norm(g1) <= 1e-4 * np.linalg.norm(g0), (np.linalg.norm(g1), np.linalg.norm(g0))
