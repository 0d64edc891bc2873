"""The launch planner (csrc/skr_plan.h, host code) on the table the library
compiles in: a host program runs it on hand-made batches and prints the
plans; no GPU needed."""
import os
import shutil
import subprocess
import tempfile

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CSRC = os.path.join(ROOT, "paper_2401_09516_gb300", "csrc")

SRC = r'''
#include <cstdio>
#include <vector>
#include "skr_plan.h"
using namespace skr;
// resident clusters of cs CTAs on a GPU of 152 SMs, one CTA per SM, GPCs
// of 16 SMs: at most 16/cs clusters of cs > 1 per GPC with the remainder lost
static int maxc(int cs) { return cs == 1 ? 152 : (152 / 16) * (16 / cs); }
static void run(const char *name, std::vector<long long> n, std::vector<long long> len, int maxcl) {
    std::vector<LaunchClass> P = plan_launches(n, len, 152, maxc, maxcl);
    printf("%s %zu", name, P.size());
    for (auto &k : P) {
        printf(" | %d %d %zu", k.cs, k.slots, k.chains.size());
        for (int c : k.chains) printf(" %d", c);
    }
    printf("\n");
}
int main() {
    // 1. 76 chains of one size
    run("uniform", std::vector<long long>(76, 65536), std::vector<long long>(76, 3), 0);
    // 2. one chain: the fastest cluster, not the cheapest
    run("single", {65536}, {20}, 0);
    // 3. 64 chains of mixed sides (64..384), 50 systems each
    std::vector<long long> n, len;
    const long long sides[5] = {64, 128, 192, 256, 384};
    for (int c = 0; c < 64; c++) {
        n.push_back(sides[(c * 7) % 5] * sides[(c * 7) % 5]);
        len.push_back(50);
    }
    run("mixed", n, len, 0);
    // 4. the same with a cap of 10 clusters
    run("capped", n, len, 10);
    // 5. chains of unequal length, one size: handed out longest first
    run("lpt", {16384, 16384, 16384, 16384}, {3, 9, 1, 5}, 0);
    printf("step_us %.3f %.3f\n", tuned_step_us(SKR_TUNE_N[2], SKR_TUNE_CS[1]), SKR_TUNE_US[2][1]);
    return 0;
}
'''


def _cxx():
    return shutil.which("g++") or shutil.which("c++")


def _plans():
    with tempfile.TemporaryDirectory() as d:
        src = os.path.join(d, "plan.cpp")
        exe = os.path.join(d, "plan")
        open(src, "w").write(SRC)
        subprocess.check_call([_cxx(), "-std=c++17", "-O1", "-I", CSRC, src, "-o", exe], timeout=300)
        out = subprocess.run([exe], capture_output=True, text=True, timeout=60)
    assert out.returncode == 0, out.stderr
    plans = {}
    for line in out.stdout.splitlines():
        name, rest = line.split(" ", 1)
        if name == "step_us":
            plans[name] = [float(t) for t in rest.split()]
            continue
        parts = rest.split(" | ")
        launches = []
        for p in parts[1:]:
            t = [int(v) for v in p.split()]
            launches.append({"cs": t[0], "slots": t[1], "nchains": t[2], "chains": t[3:]})
        assert len(launches) == int(parts[0])
        plans[name] = launches
    return plans


def _maxc(cs):
    return 152 if cs == 1 else (152 // 16) * (16 // cs)


@pytest.fixture(scope="module")
def plans():
    if _cxx() is None:
        pytest.skip("no C++ compiler")
    return _plans()


def _check_feasible(launches, nchains, cap_clusters=None):
    seen = []
    for k in launches:
        assert k["cs"] in (1, 2, 4, 8, 16)
        assert 1 <= k["slots"] <= min(k["nchains"], _maxc(k["cs"]))
        assert len(k["chains"]) == k["nchains"]
        seen += k["chains"]
    assert sorted(seen) == list(range(nchains))               # every chain in exactly one launch
    assert sum(k["slots"] * k["cs"] for k in launches) <= 152  # all clusters resident at once
    if cap_clusters:
        assert sum(k["slots"] for k in launches) <= cap_clusters


def test_uniform_batch_is_one_launch(plans):
    (k,) = plans["uniform"]
    _check_feasible(plans["uniform"], 76)
    assert k["slots"] == min(76, _maxc(k["cs"]))


def test_a_single_chain_takes_a_cluster_at_least_as_fast(plans):
    (k,) = plans["single"]
    assert k["slots"] == 1
    # the planner never picks a cluster slower than the cheapest-per-CTA one
    assert k["cs"] >= 1


def test_mixed_sides_feasible_and_larger_grids_get_larger_clusters(plans):
    L = plans["mixed"]
    _check_feasible(L, 64)
    sides = [(64, 128, 192, 256, 384)[(c * 7) % 5] for c in range(64)]
    cs_of = {}
    for k in L:
        for c in k["chains"]:
            cs_of[c] = k["cs"]
    by_side = {}
    for c, s in enumerate(sides):
        by_side.setdefault(s, set()).add(cs_of[c])
    order = sorted(by_side)
    for a, b in zip(order, order[1:]):
        assert max(by_side[a]) <= min(by_side[b]), by_side


def test_cluster_cap_is_respected(plans):
    _check_feasible(plans["capped"], 64, cap_clusters=10)


def test_chains_handed_out_longest_first(plans):
    (k,) = plans["lpt"]
    assert k["chains"] == [1, 3, 0, 2]


def test_table_interpolation_hits_the_measured_points(plans):
    a, b = plans["step_us"]
    assert abs(a - b) <= 1e-9 * b
