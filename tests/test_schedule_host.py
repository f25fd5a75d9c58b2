"""Host checks of the persistent kernels' task orders (csrc/schedule.h) and the pipeline-lag
rule (csrc/ctx.h), compiled with the host C++ compiler from the same headers the kernels use.

For the two-pass order (lag D < R slots) and the three-pass order of the adjoint (lag D,
R >= 2D + 1 slots), over many shapes:
  * every (batch, pass, index) is one task, exactly once;
  * every wait is on tasks earlier in the list (so a fully resident grid cannot deadlock);
  * a simulated persistent launch (CTA b runs tasks b, b + grid, ...; at every step a random
    CTA whose wait is met runs its task) always finishes, and whenever a task runs, the batch
    it reads is complete and the slot's next user has not overwritten it yet.
No GPU needed."""
import os
import shutil
import subprocess

import pytest

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(os.path.dirname(HERE), "paper_2601_07824_gb300", "csrc")
CUDA_INC = "/usr/local/cuda/include"

PROGRAM = r"""
#include <cstdio>
#include <cstdlib>
#include <random>
#include <vector>
#include "schedule.h"
#include "ctx.h"
using namespace hm;

static int fails = 0;
#define CHECK(c, ...) do { if (!(c)) { if (fails++ < 20) { std::printf(__VA_ARGS__); std::printf("\n"); } } } while (0)

// passes: 2 (two-pass) or 3 (adjoint); returns tasks in the list
struct Order {
    int passes, p[4], R, D;
    int64_t nb;
    int64_t total() const {
        return passes == 2 ? nb * (p[1] + p[2]) : (nb + 2 * D) * (int64_t)(p[1] + p[2] + p[3]);
    }
    // kind 0: nothing to do (three-pass stages outside [0, nb))
    void decode(int64_t t, int64_t& g, int& kind, int& r) const {
        if (passes == 2) { twopass_decode(t, p[1], p[2], nb, D, g, kind, r); return; }
        g3_decode(t, p[1], p[2], p[3], D, kind, g, r);
        if (g < 0 || g >= nb) kind = 0;
    }
    int dep(int64_t g, int kind, int& slot, unsigned& need) const {
        if (passes == 2) return twopass_dependency(g, kind, R, p[1], p[2], slot, need);
        return g3_dependency(g, kind, R, p[1], p[2], p[3], slot, need);
    }
};

static void check(const Order& o, int grid, std::mt19937& rng) {
    const int64_t T = o.total();
    const int last = o.passes;
    std::vector<int64_t> bat(T);
    std::vector<int> kd(T), rr(T);
    std::vector<std::vector<int>> seen(o.nb, std::vector<int>(16, 0));
    for (int64_t t = 0; t < T; ++t) {
        o.decode(t, bat[t], kd[t], rr[t]);
        if (kd[t] == 0) continue;
        CHECK(bat[t] >= 0 && bat[t] < o.nb && rr[t] >= 0 && rr[t] < o.p[kd[t]], "bad decode t=%lld", (long long)t);
        if (bat[t] >= 0 && bat[t] < o.nb && rr[t] >= 0 && rr[t] < o.p[kd[t]]) seen[bat[t]][kd[t]]++;
    }
    for (int64_t g = 0; g < o.nb; ++g)
        for (int k = 1; k <= o.passes; ++k)
            CHECK(seen[g][k] == o.p[k], "coverage: batch %lld pass %d seen %d of %d", (long long)g, k, seen[g][k], o.p[k]);
    // completions per (pass, slot) among tasks earlier in the list
    std::vector<std::vector<unsigned>> cnt(4, std::vector<unsigned>(o.R, 0));
    for (int64_t t = 0; t < T; ++t) {
        if (kd[t] == 0) continue;
        int slot; unsigned need;
        const int w = o.dep(bat[t], kd[t], slot, need);
        if (w) CHECK(cnt[w][slot] >= need, "wait on a later task: t=%lld", (long long)t);
        cnt[kd[t]][bat[t] % o.R]++;
    }
    // simulated persistent launch
    std::vector<int64_t> cur(grid);
    for (int b = 0; b < grid; ++b) cur[b] = b;
    std::vector<std::vector<unsigned>> c(4, std::vector<unsigned>(o.R, 0));
    std::vector<std::vector<int>> done(o.nb, std::vector<int>(4, 0));
    int64_t left = T;
    std::vector<int> ready;
    while (left > 0) {
        ready.clear();
        for (int b = 0; b < grid; ++b) {
            if (cur[b] >= T) continue;
            const int64_t t = cur[b];
            if (kd[t] == 0) { ready.push_back(b); continue; }
            int slot; unsigned need;
            const int w = o.dep(bat[t], kd[t], slot, need);
            if (!w || c[w][slot] >= need) ready.push_back(b);
        }
        if (ready.empty()) { CHECK(false, "deadlock with %lld tasks left", (long long)left); return; }
        const int b = ready[rng() % ready.size()];
        const int64_t t = cur[b];
        cur[b] += grid;
        --left;
        if (kd[t] == 0) continue;
        const int64_t g = bat[t];
        const int k = kd[t];
        // what the task reads is complete, and the slot's next user has not started writing
        if (k > 1) CHECK(done[g][k - 1] == o.p[k - 1], "pass %d of batch %lld ran before pass %d finished", k, (long long)g, k - 1);
        if (g + o.R < o.nb) CHECK(done[g + o.R][1] == 0, "slot of batch %lld reused while pass %d still reads it", (long long)g, k);
        if (k == 1 && g >= o.R) CHECK(done[g - o.R][last] == o.p[last], "batch %lld overwrote a slot still in use", (long long)g);
        done[g][k]++;
        c[k][g % o.R]++;
    }
}

int main() {
    std::mt19937 rng(12345);
    int cases = 0;
    for (int64_t nb : {1, 2, 3, 5, 8, 17})
        for (int p1 : {1, 3, 8})
            for (int p2 : {1, 2, 5})
                for (int R : {2, 3, 4, 7})
                    for (int D = 1; D < R; ++D)
                        for (int grid : {1, 3, 16}) {
                            Order o{2, {0, p1, p2, 0}, R, D, nb};
                            check(o, grid, rng);
                            ++cases;
                        }
    for (int64_t nb : {1, 2, 4, 9, 16})
        for (int p1 : {1, 4})
            for (int p2 : {1, 3})
                for (int p3 : {1, 2})
                    for (int D : {1, 2, 3})
                        for (int extra : {0, 1, 3})
                            for (int grid : {1, 5, 24}) {
                                Order o{3, {0, p1, p2, p3}, 2 * D + 1 + extra, D, nb};
                                check(o, grid, rng);
                                ++cases;
                            }
    // the pipeline-lag rule: the smallest lag with >= 1.5 grid rounds of tasks between
    // dependent passes, lowered only to fit the ring (slots of slot_bytes) and the counters
    for (int64_t per : {1, 7, 32, 64, 128, 256, 1000, 100000})
        for (int grid : {1, 152, 304})
            for (int mult : {1, 2})
                for (size_t slot : {(size_t)1 << 20, (size_t)8 << 20, (size_t)32 << 20})
                    for (size_t mx : {(size_t)64 << 20, (size_t)96 << 20}) {
                        const int D = pipeline_lag(per, grid, mult, slot, mx);
                        const bool fits = (size_t)(mult * D + 1) * slot <= mx && mult * D + 1 <= 63;
                        CHECK(D >= 1, "lag < 1");
                        CHECK(D == 1 || fits, "ring too large: per=%lld D=%d", (long long)per, D);
                        if (2 * D * per < 3 * (int64_t)grid) {  // short of 1.5 rounds: D + 1 must not fit
                            const bool fits1 = (size_t)(mult * (D + 1) + 1) * slot <= mx && mult * (D + 1) + 1 <= 63;
                            CHECK(!fits1, "lag not raised: per=%lld grid=%d D=%d", (long long)per, grid, D);
                        } else if (D > 1) {  // minimal
                            CHECK(2 * (int64_t)(D - 1) * per < 3 * (int64_t)grid, "lag not minimal: per=%lld D=%d", (long long)per, D);
                        }
                        ++cases;
                    }
    std::printf("cases %d fails %d\n", cases, fails);
    return fails ? 1 : 0;
}
"""


@pytest.fixture(scope="module")
def binary(tmp_path_factory):
    cxx = shutil.which("g++") or shutil.which("c++")
    if cxx is None:
        pytest.skip("no host C++ compiler")
    if not os.path.isdir(CUDA_INC):
        pytest.skip("no CUDA headers")
    d = tmp_path_factory.mktemp("sched")
    src, exe = d / "sched.cpp", d / "sched"
    src.write_text(PROGRAM)
    r = subprocess.run([cxx, "-O2", "-std=c++17", "-I", CSRC, "-I", CUDA_INC, str(src), "-o", str(exe)],
                       capture_output=True, text=True)
    assert r.returncode == 0, r.stderr
    return str(exe)


def test_task_orders_and_lag_rule(binary):
    r = subprocess.run([binary], capture_output=True, text=True, timeout=300)
    assert r.returncode == 0, r.stdout + r.stderr
    assert "fails 0" in r.stdout


def test_planted_mistake_is_caught(tmp_path):
    # a lag of D in the three-pass order with only 2D slots lets pass 1 of batch g + R overwrite
    # a slot that pass 3 of batch g still reads: the checker must say so
    cxx = shutil.which("g++") or shutil.which("c++")
    if cxx is None or not os.path.isdir(CUDA_INC):
        pytest.skip("no host C++ compiler or CUDA headers")
    prog = PROGRAM.replace("Order o{3, {0, p1, p2, p3}, 2 * D + 1 + extra, D, nb};",
                           "Order o{3, {0, p1, p2, p3}, 2 * D + extra, D, nb};")
    assert prog != PROGRAM
    src, exe = tmp_path / "bad.cpp", tmp_path / "bad"
    src.write_text(prog)
    r = subprocess.run([cxx, "-O2", "-std=c++17", "-I", CSRC, "-I", CUDA_INC, str(src), "-o", str(exe)],
                       capture_output=True, text=True)
    assert r.returncode == 0, r.stderr
    r = subprocess.run([str(exe)], capture_output=True, text=True, timeout=300)
    assert r.returncode != 0 and "fails 0" not in r.stdout
