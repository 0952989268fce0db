// Prints the banded Cholesky's task list (ba_band_sched.h) for the tests:
//   band_schedule nb bwt s_upd workers crit_workers [sim_max]
// first line "ncrit N", then one task per line: x y z w.
#include <cstdio>
#include <cstdlib>

#include "ba_band_sched.h"

int main(int argc, char** argv) {
  if (argc != 6 && argc != 7) {
    std::fprintf(stderr, "usage: band_schedule nb bwt s_upd workers crit_workers [sim_max]\n");
    return 2;
  }
  int ncrit = 0;
  const long long sim_max = argc == 7 ? std::atoll(argv[6]) : ba::BAND_SIM_MAX_TASKS;
  const std::vector<ba::BandTask> t =
      ba::band_tasks(std::atoi(argv[1]), std::atoi(argv[2]), std::atoi(argv[3]), std::atoi(argv[4]),
                     std::atoi(argv[5]), &ncrit, sim_max);
  std::printf("ncrit %d\n", ncrit);
  for (const ba::BandTask& q : t) std::printf("%d %d %d %d\n", q.x, q.y, q.z, q.w);
  return 0;
}
