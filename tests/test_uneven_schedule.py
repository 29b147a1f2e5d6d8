"""The uneven batch's forward schedule (csrc/uneven_schedule.h, host C++), compiled on its own with
g++ and checked on the host: the team sizes follow the stated rule, every signal is scheduled exactly
once, a team's members are distinct CTAs holding ranks 0..T-1, and the per-CTA task lists can all
run to completion when a team task starts only once every member has reached it (no cycle of
waits), for random and adversarial band-limit mixes and grid sizes."""
import ctypes
import os
import shutil
import subprocess

import numpy as np
import pytest

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(os.path.dirname(HERE), "paper_1403_4661_gb300", "csrc")

HARNESS = r'''
#include "uneven_schedule.h"
extern "C" int schedule(int n, const int *Ls, const int *lpt, int grid, int *tasks4, int cap,
                        int *start, int *small, int *nsmall, int *nteams) {
    std::vector<int> L(Ls, Ls + n), order(lpt, lpt + n), ts, sm;
    std::vector<sht::UTask> t;
    sht::plan_teams(L, order, grid, t, ts, sm, *nteams);
    if ((int)t.size() > cap) return -1;
    for (size_t i = 0; i < t.size(); ++i) {
        tasks4[4 * i] = t[i].sig; tasks4[4 * i + 1] = t[i].rank;
        tasks4[4 * i + 2] = t[i].T; tasks4[4 * i + 3] = t[i].team;
    }
    for (size_t i = 0; i < ts.size(); ++i) start[i] = ts[i];
    for (size_t i = 0; i < sm.size(); ++i) small[i] = sm[i];
    *nsmall = (int)sm.size();
    return (int)t.size();
}
'''


@pytest.fixture(scope="module")
def lib(tmp_path_factory):
    if shutil.which("g++") is None:
        pytest.skip("g++ not available")
    d = tmp_path_factory.mktemp("sched")
    src, so = os.path.join(d, "h.cpp"), os.path.join(d, "libsched.so")
    with open(src, "w") as f:
        f.write(HARNESS)
    subprocess.run(["g++", "-O1", "-std=c++17", "-shared", "-fPIC", "-I", CSRC, src, "-o", so], check=True)
    return ctypes.CDLL(so)


def _schedule(lib, Ls, grid):
    n = len(Ls)
    Ls = np.asarray(Ls, dtype=np.int32)
    lpt = np.array(sorted(range(n), key=lambda i: -int(Ls[i])), dtype=np.int32)   # stable, descending L
    cap = 16 * n + 1
    tasks = np.zeros(4 * cap, dtype=np.int32)
    start = np.zeros(grid + 1, dtype=np.int32)
    small = np.zeros(max(n, 1), dtype=np.int32)
    nsmall, nteams = ctypes.c_int(), ctypes.c_int()
    P = ctypes.POINTER(ctypes.c_int)
    ntask = lib.schedule(n, Ls.ctypes.data_as(P), lpt.ctypes.data_as(P), grid, tasks.ctypes.data_as(P), cap,
                         start.ctypes.data_as(P), small.ctypes.data_as(P), ctypes.byref(nsmall), ctypes.byref(nteams))
    assert ntask >= 0
    return lpt, tasks[:4 * ntask].reshape(-1, 4), start, small[:nsmall.value], nteams.value


def _check(lib, Ls, grid):
    lpt, tasks, start, small, nteams = _schedule(lib, Ls, grid)
    n = len(Ls)
    share = sum(float(L) ** 3 for L in Ls) / grid
    want_T = {i: min(16, int(np.floor(float(Ls[i]) ** 3 / share)), grid) if Ls[i] >= 64 else 1 for i in range(n)}
    # per-CTA lists
    lists = [tasks[start[c]:start[c + 1]] for c in range(grid)]
    assert start[grid] == len(tasks)
    members = {}
    for c, lst in enumerate(lists):
        teams = [int(t[3]) for t in lst]
        assert teams == sorted(teams) and len(set(teams)) == len(teams)   # dealt order, once per CTA
        for sig, rank, T, team in lst:
            members.setdefault(team, []).append((int(c), int(sig), int(rank), int(T)))
    assert sorted(members) == list(range(nteams))
    scheduled = []
    for team, mem in members.items():
        sigs = {m[1] for m in mem}
        Ts = {m[3] for m in mem}
        assert len(sigs) == 1 and len(Ts) == 1
        T = Ts.pop()
        assert sorted(m[2] for m in mem) == list(range(T))            # ranks 0..T-1
        assert len({m[0] for m in mem}) == T                          # distinct CTAs
        sig = sigs.pop()
        assert T == want_T[sig] and T >= 2
        scheduled.append(sig)
    # the rest run one CTA each, in descending L
    assert list(small) == [i for i in lpt if want_T[i] < 2]
    assert sorted(scheduled + list(small)) == list(range(n))
    assert _runs_to_completion([[int(t[3]) for t in lst] for lst in lists]), "the team schedule can deadlock"


def _runs_to_completion(lists):
    """Per-CTA lists of team indices: repeatedly run a team whose members all stand at it (a team
    task starts only once every member has reached it); False if no team can start while tasks
    remain (a cycle of waits)."""
    members = {}
    for c, lst in enumerate(lists):
        for team in lst:
            members.setdefault(team, []).append(c)
    head = [0] * len(lists)
    left = sum(len(lst) for lst in lists)
    while left:
        progressed = False
        for team, mem in members.items():
            if all(head[c] < len(lists[c]) and lists[c][head[c]] == team for c in mem):
                for c in mem:
                    head[c] += 1
                left -= len(mem)
                progressed = True
        if not progressed:
            return False
    return True


def test_the_deadlock_check_has_teeth():
    assert _runs_to_completion([[0, 1], [0, 1], [1]])
    assert not _runs_to_completion([[0, 1], [1, 0]])          # two CTAs taking two teams in opposite order


@pytest.mark.parametrize("grid", [1, 2, 7, 152, 304])
def test_loguniform_batches(lib, grid):
    rng = np.random.default_rng(grid)
    for n in (1, 5, 64, 512):
        Ls = np.rint(np.exp(rng.uniform(np.log(32), np.log(1024), n))).astype(int)
        _check(lib, Ls, grid)


@pytest.mark.parametrize("Ls", [[1024] * 40, [1024, 1023, 900, 64, 63, 2, 1], [64] * 300 + [1000] * 3,
                                [2048] + [32] * 100, [512] * 152])
def test_adversarial_batches(lib, Ls):
    for grid in (3, 16, 17, 152, 304):
        _check(lib, Ls, grid)


def test_the_rule_on_a_known_batch(lib):
    # one dominant signal: its chain is most of the work, so it gets the full team of 16
    lpt, tasks, start, small, nteams = _schedule(lib, [1000] + [100] * 50, 152)
    assert nteams == 1 and {int(t[2]) for t in tasks} == {16} and len(small) == 50
