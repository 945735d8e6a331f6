"""Host logic of bench.py (CPU only): the clock record keeps only samples
taken inside the timed region, the reference arm sizes each step's sample so
warm-up plus timed steps stay within its time budget, and the end-to-end leg's
batched calls cover the steps without running across a trajectory restart."""
import argparse

import pytest

import bench


def _line(sm, smax, active=("Not Active",) * 4):
    return "0, %s, %s, 900.0, 0x0, %s\n" % (sm, smax, ", ".join(active))


def test_clock_summary_keeps_the_timed_region_only():
    lines = [(0.5, _line(1000, 2070)),  # before the region (idle clock)
             (1.1, _line(2070, 2070)), (1.2, _line(2065, 2070)),
             (1.3, _line(2070, 2070, ("Not Active", "Not Active", "Not Active", "Active"))),
             (2.5, _line(800, 2070))]  # after
    c = bench.ClockSampler.summarize(lines, 1.0, 2.0)
    assert c["samples"] == 3 and c["sm_mhz"] == 2070.0 and c["sm_max_mhz"] == 2070.0
    assert c["reasons"] == ["sw_power_cap"]
    empty = bench.ClockSampler.summarize(lines, 3.0, 3.05)
    assert empty["samples"] == 0 and empty["sm_mhz"] is None
    near = bench.ClockSampler.summarize(lines, 2.6, 2.65)  # no sample inside: the one at 2.5 s stands in
    assert near["samples"] == 1 and near["sm_mhz"] == 800.0 and near["adjacent"]


def test_clock_summary_skips_malformed_lines():
    lines = [(1.1, "garbage\n"), (1.2, "0, [N/A], 2070, 1, 0x0, a, b, c, d\n"), (1.3, _line(1900, 2070))]
    c = bench.ClockSampler.summarize(lines, 1.0, 2.0)
    assert c["samples"] == 1 and c["sm_mhz"] == 1900.0


class _FakeOracle:
    """Stands in for the oracle: each call costs cells * iterations / rate on a fake clock."""

    def __init__(self, clock, rate):
        self.clock, self.rate = clock, rate
        self.cells = []

    def Problem(self, prob):
        return prob

    def run(self, P, method, n_steps, tol, max_iter, commit_unconverged):
        self.cells.append(P["n_cells"])
        self.clock[0] += P["n_cells"] * max_iter / self.rate

    def max_threads(self):
        return 16


def _args(steps, warmup, workload="slab", cells=65536):
    return argparse.Namespace(gpus=1, steps=steps, warmup=warmup, impl="reference", workload=workload,
                              precision="fp32", n_ord=64, cells=cells, c=0.9, dx=0.1, seed=4, nn_seed=101)


def _run_reference(monkeypatch, steps, warmup, rate, **kw):
    import sys
    clock = [0.0]
    fake = _FakeOracle(clock, rate)
    monkeypatch.setitem(sys.modules, "oracle", fake)
    monkeypatch.setattr(bench.time, "perf_counter", lambda: clock[0])
    r = bench.run_reference(_args(steps, warmup, **kw), budget_s=150.0)
    return r, clock[0], fake


def test_reference_arm_runs_two_iterations_of_the_whole_problem_when_they_fit(monkeypatch):
    r, total, fake = _run_reference(monkeypatch, steps=20, warmup=3, rate=65536 / 0.2)  # 0.2 s per iteration
    assert set(fake.cells) == {65536}
    assert "2 OCI iteration(s) per step of the 65536-cell" in r["cpu_baseline"]["sample"]
    assert abs(r["value"] - 65536 * 64 / 0.2) < 1e-6 * r["value"]
    assert total < 150.0


def test_reference_arm_scales_the_slab_down_for_many_steps(monkeypatch):
    r, total, fake = _run_reference(monkeypatch, steps=1000, warmup=5, rate=65536 / 0.2)
    js = fake.cells[-1]
    assert js < 65536 and js % 256 == 0 and js >= 1024
    assert f"a {js}-cell slab" in r["cpu_baseline"]["sample"]
    assert total < 1.1 * 150.0  # warm-up and timed steps within the budget (plus the probe)
    assert abs(r["value"] - 65536 * 64 / 0.2) < 1e-6 * r["value"]  # the same rate, measured on the smaller slab
    assert r["e2e"]["value"] == r["value"] and r["impl"] == "reference"


def test_reference_arm_on_the_default_layered_slab(monkeypatch):
    """The default workload (cells = 0: the 131072-cell layered slab) with the
    driver's step counts: two iterations of the whole problem per step fit."""
    r, total, fake = _run_reference(monkeypatch, steps=20, warmup=5, rate=131072 / 0.5, workload="hetero", cells=0)
    assert set(fake.cells) == {131072}
    assert "131072-cell S_64" in r["cpu_baseline"]["sample"] and "layered slab" in r["config"]["workload"]
    assert total < 150.0


@pytest.mark.parametrize("k0,steps,n_traj,ch", [(1005, 1000, 100, 32), (25, 20, 100, 32), (0, 7, 3, 2),
                                               (100, 100, 100, 32), (99, 3, 100, 32)])
def test_end_to_end_calls_cover_the_steps_without_crossing_a_restart(k0, steps, n_traj, ch):
    """The end-to-end leg's calls of oci_run_steps: exactly `steps` steps, at
    most ch per call, a restart from psi0 before a call exactly when the
    trajectory is at a multiple of its length (and not at its very start), and
    no call running across a trajectory's end."""
    calls = bench.trajectory_chunks(k0, steps, n_traj, ch)
    assert sum(m for _, m in calls) == steps
    k = k0
    for restart, m in calls:
        assert 1 <= m <= ch
        assert restart == (k > 0 and k % n_traj == 0)
        assert k // n_traj == (k + m - 1) // n_traj  # inside one pass over the trajectory
        k += m
