// Host side of the banded Cholesky (ba_band.cuh): the task list and its
// order.  Plain C++ (no CUDA), so that the schedule can be checked on a
// host: tests/c/band_schedule.cpp prints it, and the tests execute it.
#pragma once

#include <algorithm>
#include <functional>
#include <queue>
#include <utility>
#include <vector>

namespace ba {

// Task types (ba_band.cuh): D the diagonal chain, U an update, T a tile's
// solve, F / B the forward / backward block solves, I a diagonal tile's
// inverse transpose.
enum { BAND_D = 0, BAND_U = 1, BAND_T = 2, BAND_F = 3, BAND_B = 4, BAND_I = 5 };
constexpr int BAND_CRIT_BLOCKS = 4;             // blocks of the near-diagonal pool
constexpr long long BAND_SIM_MAX_TASKS = 2000000;  // longest list that is simulated

// One task, as the device reads it (an int4): x = type + 8 count (count:
// U's columns), y = I, z = J, w = Ka (U's first column); for D, I, F:
// y = z = J; for B: y = z = I.
struct BandTask {
  int x, y, z, w;
};

// The banded Cholesky's tasks in ticket order.
//  1. A topological enumeration by step s = 0 .. nb - 1: D_s; I_s; the update
//     segments whose last column is s - 1; the solves T(I, s); F_s; then
//     B_{nb-1} .. B_0.  Each task's predecessors are listed; D_J's
//     subdiagonal tile L_{J,J-1} is published early (after its solve, before
//     the update and factorisation of L_JJ).
//  2. Each task's longest path to the end (its priority), from rough
//     durations in microseconds (D 20, of which 8 before the early output;
//     U 12 per column; T 7; I 8; F and B 4; 1 per dependency).
//  3. A list-scheduling simulation on `workers` blocks: a free block takes
//     the ready task of highest priority.  The tickets follow the simulated
//     start times.  A task starts after its predecessors' outputs, which
//     come after their starts, so the order is topological.
// s_upd: columns per update segment; workers blocks in all, crit_workers
// of them for the near-diagonal pool; *ncrit: that pool's tasks (the list's
// first ones).  A list of more than sim_max tasks is returned in the
// enumeration's order (topological), in one pool (*ncrit = 0).
inline std::vector<BandTask> band_tasks(int nb, int bwt, int s_upd, int workers, int crit_workers, int* ncrit,
                                        long long sim_max = BAND_SIM_MAX_TASKS) {
  const long long ntile = (long long)nb * (bwt + 1);
  auto k0 = [&](int I) { return std::max(0, I - bwt); };
  auto tix = [&](int I, int J) { return (long long)J * (bwt + 1) + (I - J); };
  auto kend = [&](int I, int J) { return I == J ? J - 1 : J; };  // (J, J) leaves K = J - 1 to D_J
  std::vector<long long> seg0(ntile + 1, 0);
  for (int J = 0; J < nb; ++J)
    for (int I = J; I < std::min(nb, J + bwt + 1); ++I) {
      const int u = std::max(0, kend(I, J) - k0(I));
      seg0[tix(I, J) + 1] = (u + s_upd - 1) / s_upd;
    }
  for (long long t = 0; t < ntile; ++t) seg0[t + 1] += seg0[t];
  // a list too long to simulate keeps the enumeration's order, in one pool
  const bool simulate = seg0[ntile] + 6LL * nb <= sim_max;
  if (!simulate) crit_workers = 0;
  std::vector<int> segid(seg0[ntile], -1), idD(nb), idI(nb), idF(nb), idB(nb), idT(ntile, -1);
  std::vector<BandTask> task;
  std::vector<double> dur;
  std::vector<int> pbeg(1, 0), pred;  // predecessors: id * 2 + (1: D's early output)
  auto prod = [&](int I, int K) {
    return I == K ? 2 * idD[K] : (I == K + 1 ? 2 * idD[K + 1] + 1 : 2 * idT[tix(I, K)]);
  };
  auto last_seg = [&](int I, int J) {
    const long long t = tix(I, J);
    return seg0[t + 1] > seg0[t] ? segid[seg0[t + 1] - 1] : -1;
  };
  auto dep = [&](int p2) {
    if (p2 >= 0 && simulate) pred.push_back(p2);
  };
  auto add = [&](int type, int cnt, int I, int J, int Ka, double d) {
    task.push_back(BandTask{type + 8 * cnt, I, J, Ka});
    dur.push_back(d);
    pbeg.push_back((int)pred.size());
    return (int)task.size() - 1;
  };
  for (int st = 0; st < nb; ++st) {
    if (st >= 1) {
      dep(2 * idD[st - 1]);
      if (bwt >= 1) {
        const int a = last_seg(st, st - 1), b = last_seg(st, st);
        if (a >= 0) dep(2 * a);
        if (b >= 0) dep(2 * b);
      }
    }
    idD[st] = add(BAND_D, 0, st, st, 0, 20.0);
    dep(2 * idD[st]);
    idI[st] = add(BAND_I, 0, st, st, 0, 8.0);
    for (int J = st; J < std::min(nb, st + bwt); ++J)
      for (int I = J; I < std::min(nb, st + bwt); ++I) {
        const int K = st - 1, a0 = k0(I), e = kend(I, J);
        if (K < a0 || K >= e) continue;
        if ((K - a0 + 1) % s_upd != 0 && K != e - 1) continue;
        const int m = (K - a0) / s_upd, Ka = a0 + m * s_upd;
        if (m >= 1) dep(2 * segid[seg0[tix(I, J)] + m - 1]);
        for (int k = Ka; k <= K; ++k) {
          dep(prod(I, k));
          dep(prod(J, k));
        }
        segid[seg0[tix(I, J)] + m] = add(BAND_U, st - Ka, I, J, Ka, 12.0 * (st - Ka));
      }
    for (int I = st + 2; I < std::min(nb, st + bwt + 1); ++I) {
      dep(2 * idD[st]);
      const int a = last_seg(I, st);
      if (a >= 0) dep(2 * a);
      idT[tix(I, st)] = add(BAND_T, 0, I, st, 0, 7.0);
    }
    if (st >= 1) dep(2 * idF[st - 1]);
    for (int K = k0(st); K <= st; ++K) dep(prod(st, K));
    dep(2 * idI[st]);
    idF[st] = add(BAND_F, 0, st, st, 0, 4.0);
  }
  for (int I = nb - 1; I >= 0; --I) {
    dep(2 * idF[nb - 1]);
    if (I + 1 < nb) dep(2 * idB[I + 1]);
    idB[I] = add(BAND_B, 0, I, I, 0, 4.0);
  }
  const int nt = (int)task.size();
  if (!simulate) {
    *ncrit = 0;
    return task;
  }
  const double lat = 1.0, early = 8.0;
  auto out_time = [&](int p2, double start_or_len) { return (p2 & 1) ? early : start_or_len; };
  // longest path to the end
  std::vector<double> bl(nt, 0.0);
  for (int t = nt - 1; t >= 0; --t) {
    bl[t] = std::max(bl[t], dur[t]);
    for (int k = pbeg[t]; k < pbeg[t + 1]; ++k) {
      const int p = pred[k] >> 1;
      bl[p] = std::max(bl[p], out_time(pred[k], dur[p]) + lat + bl[t]);
    }
  }
  // the near-diagonal tasks (the chain D_J and what feeds it: updates that
  // reach a tile at most two block rows below their column, the solves two
  // below the diagonal) form a pool of their own, run by `crit_workers`
  // blocks, so that they never queue behind the bulk updates
  std::vector<int> crit(nt, 0);
  for (int t = 0; t < nt && crit_workers > 0; ++t) {
    const BandTask q = task[t];
    const int type = q.x & 7;
    crit[t] = type == BAND_D || (type == BAND_U && q.y <= q.w + (q.x >> 3) - 1 + 2) ||
              (type == BAND_T && q.y == q.z + 2);
  }
  // list scheduling: at each moment the idle blocks of a pool take its ready
  // tasks, highest priority first
  std::vector<std::vector<int>> succ(nt);
  std::vector<int> npred(nt, 0);
  for (int t = 0; t < nt; ++t)
    for (int k = pbeg[t]; k < pbeg[t + 1]; ++k) {
      succ[pred[k] >> 1].push_back(t * 2 + (pred[k] & 1));
      ++npred[t];
    }
  std::vector<double> ready(nt, 0.0), start(nt, 0.0);
  typedef std::pair<double, int> E;
  std::priority_queue<E, std::vector<E>, std::greater<E>> pending, events;  // by time
  auto higher = [&](int x, int y) { return bl[x] < bl[y] || (bl[x] == bl[y] && x > y); };
  std::priority_queue<int, std::vector<int>, decltype(higher)> avail[2] = {
      std::priority_queue<int, std::vector<int>, decltype(higher)>(higher),
      std::priority_queue<int, std::vector<int>, decltype(higher)>(higher)};
  int idle[2] = {std::max(1, workers - crit_workers), crit_workers};
  for (int t = 0; t < nt; ++t)
    if (npred[t] == 0) pending.push(E(0.0, t));
  double clock = 0.0;
  int done = 0;
  while (done < nt) {
    // outputs due by now release their successors; ready tasks join their pool
    while (!events.empty() && events.top().first <= clock) {
      const int code = events.top().second;
      const double tm = events.top().first;
      events.pop();
      const int p = code >> 1, early_out = code & 1;
      if (!early_out) ++idle[crit[p]];
      for (int s2 : succ[p])
        if ((s2 & 1) == early_out) {
          const int q = s2 >> 1;
          ready[q] = std::max(ready[q], tm + lat);
          if (--npred[q] == 0) pending.push(E(ready[q], q));
        }
    }
    while (!pending.empty() && pending.top().first <= clock) {
      avail[crit[pending.top().second]].push(pending.top().second);
      pending.pop();
    }
    for (int pl = 0; pl < 2; ++pl)
      while (idle[pl] > 0 && !avail[pl].empty()) {
        const int t = avail[pl].top();
        avail[pl].pop();
        --idle[pl];
        start[t] = clock;
        events.push(E(clock + dur[t], 2 * t));
        if ((task[t].x & 7) == BAND_D) events.push(E(clock + early, 2 * t + 1));
        ++done;
      }
    double nxt = 1e300;
    if (!events.empty()) nxt = std::min(nxt, events.top().first);
    if (!pending.empty()) nxt = std::min(nxt, pending.top().first);
    if (nxt == 1e300) break;  // not reached: the enumeration is acyclic
    clock = std::max(clock, nxt);
  }
  // tickets: the critical pool's tasks, then the bulk pool's, each by
  // simulated start
  std::vector<int> order(nt);
  for (int t = 0; t < nt; ++t) order[t] = t;
  std::stable_sort(order.begin(), order.end(), [&](int x, int y) {
    return crit[x] != crit[y] ? crit[x] > crit[y] : start[x] < start[y];
  });
  *ncrit = 0;
  for (int t = 0; t < nt; ++t) *ncrit += crit[t];
  std::vector<BandTask> out(nt);
  for (int t = 0; t < nt; ++t) out[t] = task[order[t]];
  return out;
}

}  // namespace ba
