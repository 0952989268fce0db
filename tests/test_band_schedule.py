"""The banded Cholesky's schedule (csrc/ba_band_sched.h, the host side of
the pose-graph direct solver): the task list printed by a host build of
the scheduler (tests/c/band_schedule.cpp) is executed here by blocking
workers in two pools, as the cooperative launch runs it, with the waits of
the device tasks.  Checked: every task is listed once and the list covers
the factorisation and both solves; no interleaving deadlocks (completions
in random order); and the tile arithmetic of the tasks, run in that order,
gives numpy's Cholesky factor and solution of a random banded SPD system.
No GPU."""
import os
import shutil
import subprocess

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
TB = 32
D, U, T, F, B, INV = 0, 1, 2, 3, 4, 5


@pytest.fixture(scope="module")
def scheduler(tmp_path_factory):
    if shutil.which("g++") is None:
        pytest.skip("g++ not available")
    exe = tmp_path_factory.mktemp("band") / "band_schedule"
    subprocess.run(["g++", "-std=c++17", "-O2", "-Wall", "-Wextra", "-Werror", "-I",
                    os.path.join(ROOT, "paper_2409_12190_gb300", "csrc"),
                    os.path.join(ROOT, "tests", "c", "band_schedule.cpp"), "-o", str(exe)], check=True)

    def run(nb, bwt, s_upd, workers, crit, sim_max=None):
        argv = [str(exe), str(nb), str(bwt), str(s_upd), str(workers), str(crit)]
        if sim_max is not None:
            argv.append(str(sim_max))
        out = subprocess.run(argv, capture_output=True, text=True, check=True).stdout.splitlines()
        ncrit = int(out[0].split()[1])
        tasks = [tuple(int(v) for v in line.split()) for line in out[1:]]
        return ncrit, tasks
    return run


def _k0(I, bwt):
    return max(0, I - bwt)


def _expected(nb, bwt):
    """Tiles, and the update columns each tile receives from U tasks
    (the diagonal tile's last one, K = J - 1, belongs to D_J)."""
    upd = {}
    for J in range(nb):
        for I in range(J, min(nb, J + bwt + 1)):
            end = J - 1 if I == J else J
            upd[(I, J)] = list(range(_k0(I, bwt), max(_k0(I, bwt), end)))
    return upd


class Machine:
    """The device state the tasks wait on, with the tile arithmetic."""

    def __init__(self, A, b, nb, bwt):
        n = A.shape[0]
        self.n, self.nb, self.bwt, self.b = n, nb, bwt, b
        Ap = np.eye(nb * TB)
        Ap[:n, :n] = A
        self.T = {}
        for J in range(nb):
            for I in range(J, min(nb, J + bwt + 1)):
                t = Ap[I * TB:(I + 1) * TB, J * TB:(J + 1) * TB].copy()
                self.T[(I, J)] = np.tril(t) if I == J else t
        self.flag, self.prog = set(), {k: 0 for k in self.T}
        self.inv, self.rs, self.Ui = set(), {}, {}
        self.y = np.zeros(nb * TB)
        self.c1 = self.c2 = 0

    # the waits of each device task
    def ready(self, task):
        x, I, J, Ka = task
        typ, cnt, bwt, nb = x & 7, x >> 3, self.bwt, self.nb
        if typ == D:
            if J >= 1 and bwt >= 1:
                nu = J - 1 - _k0(J, bwt)
                return (J - 1, J - 1) in self.flag and self.prog[(J, J - 1)] >= nu and self.prog[(J, J)] >= nu
            return True
        if typ == U:
            return self.prog[(I, J)] >= Ka - _k0(I, bwt) and all(
                (I, K) in self.flag and (J, K) in self.flag for K in range(Ka, Ka + cnt))
        if typ == T:
            return (J, J) in self.flag and self.prog[(I, J)] >= J - _k0(I, bwt)
        if typ == INV:
            return (J, J) in self.flag
        if typ == F:
            return all((J, K) in self.flag for K in range(_k0(J, bwt), J)) and self.c1 >= J and J in self.inv
        return self.c1 >= nb and self.c2 >= nb - 1 - I

    @staticmethod
    def _trsm(A, L, rs):
        """X L^T = A: column by column with L's columns prescaled by 1 / L_cc."""
        Ls = L * rs[None, :]
        X = A.copy()
        for c in range(TB - 1):
            X[:, c + 1:] -= np.outer(X[:, c], Ls[c + 1:, c])
        return X * rs[None, :]

    @staticmethod
    def _potrf(C):
        """Right-looking with deferred column scaling; returns L and 1 / L_cc."""
        S = C.copy()
        d = np.zeros(TB)
        rs = np.zeros(TB)
        d[0], rs[0] = S[0, 0], 1.0 / np.sqrt(S[0, 0])
        for c in range(TB - 1):
            inv = rs[c] * rs[c]
            for r in range(c + 1, TB):
                S[r, c + 1:r + 1] -= (S[r, c] * inv) * S[c + 1:r + 1, c]
            d[c + 1], rs[c + 1] = S[c + 1, c + 1], 1.0 / np.sqrt(S[c + 1, c + 1])
        return np.tril(S, -1) * rs[None, :] + np.diag(d * rs), rs

    def run(self, task):
        x, I, J, Ka = task
        typ, cnt, bwt, nb = x & 7, x >> 3, self.bwt, self.nb
        if typ == D:
            C = self.T[(J, J)]
            if J >= 1 and bwt >= 1:
                X = self._trsm(self.T[(J, J - 1)], self.T[(J - 1, J - 1)], self.rs[J - 1])
                self.T[(J, J - 1)] = X
                self.flag.add((J, J - 1))
                C = C - np.tril(X @ X.T)
            self.T[(J, J)], self.rs[J] = self._potrf(C)
            self.flag.add((J, J))
        elif typ == U:
            for K in range(Ka, Ka + cnt):
                self.T[(I, J)] = self.T[(I, J)] - self.T[(I, K)] @ self.T[(J, K)].T
            self.prog[(I, J)] = Ka + cnt - _k0(I, bwt)
        elif typ == T:
            self.T[(I, J)] = self._trsm(self.T[(I, J)], self.T[(J, J)], self.rs[J])
            self.flag.add((I, J))
        elif typ == INV:
            self.Ui[J] = self._trsm(np.eye(TB), self.T[(J, J)], self.rs[J])
            self.inv.add(J)
        elif typ == F:
            part = np.zeros(TB)
            for K in range(_k0(J, bwt), J):
                part += self.T[(J, K)] @ self.y[K * TB:(K + 1) * TB]
            v = np.array([self.b[J * TB + r] if J * TB + r < self.n else 0.0 for r in range(TB)]) - part
            self.y[J * TB:(J + 1) * TB] = self.Ui[J].T @ v
            self.c1 = J + 1
        else:
            part = np.zeros(TB)
            for K in range(min(nb - 1, I + bwt), I, -1):
                part += self.T[(K, I)].T @ self.y[K * TB:(K + 1) * TB]
            self.y[I * TB:(I + 1) * TB] = self.Ui[I] @ (self.y[I * TB:(I + 1) * TB] - part)
            self.c2 = nb - I


def _execute(machine, ncrit, tasks, workers, crit, seed):
    """Two pools of blocking workers take their pool's tickets in order; a
    held task completes once its waits hold, in random order among those
    that may.  Raises on a deadlock."""
    rng = np.random.default_rng(seed)
    pools = [list(tasks[ncrit:]), list(tasks[:ncrit])]
    sizes = [workers - crit, crit] if ncrit else [workers, 0]
    nxt, held, done = [0, 0], [[], []], 0
    while done < len(tasks):
        for p in (0, 1):
            while len(held[p]) < sizes[p] and nxt[p] < len(pools[p]):
                held[p].append(pools[p][nxt[p]])
                nxt[p] += 1
        cand = [(p, k) for p in (0, 1) for k, t in enumerate(held[p]) if machine.ready(t)]
        if not cand:
            raise AssertionError(f"deadlock with {done} of {len(tasks)} tasks done")
        p, k = cand[rng.integers(len(cand))]
        machine.run(held[p].pop(k))
        done += 1


CASES = [  # nb, bwt, columns per update task, blocks, near-diagonal blocks[, longest simulated list]
    (7, 3, 1, 8, 2),
    (11, 10, 1, 16, 3),   # dense lower triangle
    (16, 5, 2, 12, 2),    # update segments of two columns
    (13, 6, 3, 5, 1),     # segments of three, few blocks
    (5, 0, 1, 4, 1),      # diagonal: no coupling
    (1, 0, 1, 2, 1),      # one block
    (20, 4, 1, 152, 4),
    (9, 8, 1, 1, 0),      # one block for everything (no near-diagonal pool)
    (10, 9, 2, 6, 2, 0),  # too long to simulate: the enumeration's order, one pool
]


def _case(c):
    return c + (None,) * (6 - len(c))


@pytest.mark.parametrize("nb,bwt,s_upd,workers,crit,sim_max", [_case(c) for c in CASES])
def test_task_list_covers_the_factorisation_once(scheduler, nb, bwt, s_upd, workers, crit, sim_max):
    ncrit, tasks = scheduler(nb, bwt, s_upd, workers, crit, sim_max)
    if sim_max == 0:
        assert ncrit == 0
    assert len(set(tasks)) == len(tasks)
    types = [t[0] & 7 for t in tasks]
    for typ in (D, INV, F, B):
        assert sorted(t[2] for t in tasks if t[0] & 7 == typ) == list(range(nb))
    got = {}
    for x, I, J, Ka in tasks:
        if x & 7 == U:
            assert 1 <= x >> 3 <= s_upd
            got.setdefault((I, J), []).extend(range(Ka, Ka + (x >> 3)))
    want = _expected(nb, bwt)
    assert {k: sorted(v) for k, v in got.items()} == {k: v for k, v in want.items() if v}
    solves = sorted((I, J) for x, I, J, _ in tasks if x & 7 == T)
    assert solves == sorted((I, J) for (I, J) in want if I >= J + 2)
    # the near-diagonal pool: D, updates at most two rows below their
    # column, solves two rows below the diagonal
    for x, I, J, Ka in tasks[:ncrit]:
        typ = x & 7
        assert typ == D or (typ == U and I <= Ka + (x >> 3) + 1) or (typ == T and I == J + 2)
    assert (ncrit == 0) == (crit == 0 or sim_max == 0) or types.count(D) == 0


@pytest.mark.parametrize("nb,bwt,s_upd,workers,crit,sim_max", [_case(c) for c in CASES])
def test_two_pool_execution_never_deadlocks_and_solves(scheduler, nb, bwt, s_upd, workers, crit, sim_max):
    ncrit, tasks = scheduler(nb, bwt, s_upd, workers, crit, sim_max)
    rng = np.random.default_rng(nb * 100 + bwt)
    n = nb * TB - 5 if nb > 1 else 20   # ragged: the padding's identity rows
    bw = min(n - 1, max(0, bwt * TB - 7))
    M = np.zeros((n, n))
    for r in range(n):
        lo = max(0, r - bw)
        M[r, lo:r + 1] = rng.standard_normal(r + 1 - lo)
    A = np.tril(np.triu(M @ M.T, -bw), bw)
    A += np.eye(n) * (np.abs(A).sum(1).max() + 1.0)
    b = rng.standard_normal(n)
    L_ref = np.linalg.cholesky(A)
    x_ref = np.linalg.solve(A, b)
    for seed in range(3):
        m = Machine(A, b, nb, bwt)
        _execute(m, ncrit, tasks, workers, crit, seed)
        Lf = np.zeros((nb * TB, nb * TB))
        for (I, J), t in m.T.items():
            Lf[I * TB:(I + 1) * TB, J * TB:(J + 1) * TB] = t
        assert np.max(np.abs(Lf[:n, :n] - L_ref)) <= 1e-13 * np.max(np.abs(L_ref))
        assert np.max(np.abs(m.y[:n] - x_ref)) <= 1e-12 * np.max(np.abs(x_ref))
