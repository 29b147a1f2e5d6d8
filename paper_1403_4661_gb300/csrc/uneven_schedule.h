// Host-side schedule of the uneven batch's forward order chains (host C++ only, no CUDA: the
// library's csrc/uneven.cu uses it at sht_uneven_create, and a CPU test compiles it on its own to
// check the schedule's invariants).
#pragma once

#include <algorithm>
#include <cmath>
#include <vector>

namespace sht {

// One member's share of a team chain: signal, rank in the team, team size, team index.
struct UTask {
    int sig, rank, T, team;
};

constexpr int kMaxTeam = 16;    // CTAs of one team chain: two team barriers per order each

// Forward phase 2's schedule.  The chain of a signal of band-limit L costs ~L^3; a signal whose
// chain exceeds two CTAs' fair share of the batch (share = sum of L^3 over the grid) runs on a
// team of T = min(16, floor(L^3 / share)) CTAs (L >= 64); the others run on one CTA each from a
// queue (`small`, in the order of `lpt`).  (Splitting every chain above half a share, into
// ceil(2 L^3 / share) members, measured slower on the 512-signal workload: more teams leave more
// CTAs waiting for team partners.)  Teams, in the order of `lpt` (largest first), take consecutive
// CTAs, wrapping to CTA 0 when the grid is used up; every CTA runs its team tasks in the order
// they were dealt (CTA c: tasks[task_start[c] .. task_start[c+1])), so a team waits only for
// members busy with earlier teams and no cycle of waits can form.
//   Ls[i]: band-limit of signal i; lpt: signal indices by descending L; grid: CTAs of the launch.
inline void plan_teams(const std::vector<int> &Ls, const std::vector<int> &lpt, int grid, std::vector<UTask> &tasks,
                       std::vector<int> &task_start, std::vector<int> &small, int &nteams) {
    double total = 0.0;
    for (int L : Ls) total += (double)L * L * L;
    const double share = grid > 0 ? total / grid : 1.0;
    std::vector<std::vector<UTask>> per((size_t)std::max(grid, 1));
    int cursor = 0;
    nteams = 0;
    for (int i : lpt) {
        const int L = Ls[(size_t)i];
        const double w = (double)L * L * L;
        int T = L >= 64 ? (int)std::min<double>(kMaxTeam, std::floor(w / share)) : 1;
        T = std::min(T, grid);
        if (T < 2) { small.push_back(i); continue; }
        if (cursor + T > grid) cursor = 0;
        for (int r = 0; r < T; ++r) per[(size_t)(cursor + r)].push_back(UTask{i, r, T, nteams});
        cursor += T;
        ++nteams;
    }
    task_start.assign((size_t)std::max(grid, 0) + 1, 0);
    for (int c = 0; c < grid; ++c) {
        task_start[(size_t)c + 1] = task_start[(size_t)c] + (int)per[(size_t)c].size();
        tasks.insert(tasks.end(), per[(size_t)c].begin(), per[(size_t)c].end());
    }
}

}  // namespace sht
