"""Host-side helpers of bench.py: the DRAM-traffic table it reads from the profiles folder, and
the count of MMA flops the tensor-core transfer build issues."""
import importlib.util
import os

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _bench():
    spec = importlib.util.spec_from_file_location("bench_mod", os.path.join(ROOT, "bench.py"))
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    return mod


def test_traffic_table_has_the_benchmarked_kernels():
    t = _bench()._traffic_table()
    assert t[("k_sbuild_tc", 2048, 32)] > 0
    # the interface apply reads every stored HODLR entry about once: ~0.17 GB per launch
    assert 0.1e9 < t[("hodlr_apply", 2048, 32)] < 0.3e9


def test_tensor_core_flop_count():
    f = _bench()._tc_executed_flops
    # a single CTA with one partly filled tile: 64 sources on 64 blocks (n = 65), MB = 32
    nb, MB = 64, 32
    up = nb - 1      # upward sweep from block 64: 63 steps
    down = nb - 1    # downward sweep from block 1: 63 steps
    assert f(1, nb, MB) == (up + down) * 3 * 2 * 128 * MB * MB
    # every source visits every other block once: the executed work covers the algorithmic
    # (m x m) x (m x 1) products at least three times over (3xTF32), on padded blocks
    nds, nb, m = 63, 2047, 63
    assert f(nds, nb, 64) >= 3 * nds * nb * (nb - 1) * 2.0 * m * m


def test_clock_log_summary():
    """Median and maximum SM clock and the throttle reasons of an nvidia-smi sample log."""
    S = _bench().ClockSampler.summarize
    q = "0, {sm}, 2070, 900.5, 0x0000000000000000, Not Active, Not Active, Not Active, {cap}"
    lines = [q.format(sm=sm, cap=cap) for sm, cap in
             [(2070, "Not Active"), (1980, "Active"), (2055, "Not Active")]]
    lines.append("0, [N/A], 2070, 0, 0x0, Not Active, Not Active, Not Active, Not Active")
    lines.append("garbled")
    r = S(lines)
    assert r == {"sm_mhz": 2055.0, "sm_max_mhz": 2070.0, "reasons": ["sw_power_cap"], "samples": 3}
    hot = "0, 1500, 2070, 1400, 0x8, Active, Not Active, Active, Not Active"
    assert S([hot])["reasons"] == ["hw_slowdown", "sw_thermal_slowdown"]
    assert S([])["sm_mhz"] is None and S([])["samples"] == 0


def test_cpu_baseline_reports_busy_threads():
    """The oracle baseline reports its rate, the host's cores and the threads it kept busy."""
    r = _bench().cpu_baseline(n=64)
    assert r["kind"] == "oracle" and r["unit"] == "DOF/s" and r["value"] > 0
    assert r["cores"] == os.cpu_count()
    assert 0.0 < r["threads_busy"] <= r["cores"] + 0.5


def test_reference_sample_size_is_bounded_by_the_step_count():
    size = _bench()._ref_size
    assert size(5, 3) == 512 and size(7, 3) == 512     # default run: about two minutes
    assert size(20, 3) == 256                          # longer runs take the smaller sample
    assert size(20, 3, 128) == 128                     # an explicit size wins


def test_cpu_leg_reports_errors_of_both_solutions():
    """The CPU leg measures the timed run's solution and the HBS section's solution against
    the oracle's global solve of the same instance (exact solutions give zero, a perturbed one
    its relative size)."""
    import numpy as np

    import ddst_inputs as I
    from oracle import ddst_oracle as O
    prob = I.make_problem("convdiff2d", n=64, w=16)
    A, b = O.assemble(prob)
    ustar = O.global_solve(A, b)
    pert = ustar.reshape(63, 63) * (1.0 + 1e-6)
    leg = _bench().cpu_leg(prob, ustar.copy(), verify=True, ref_n=64, u_hbs=pert)
    assert leg["verify"]["rel_error_vs_oracle"] <= 1e-14
    assert abs(leg["hbs_rel_error_vs_oracle"] - 1e-6) <= 1e-9
    assert leg["cpu_baseline"]["kind"] == "oracle"
    leg = _bench().cpu_leg(prob, ustar.copy(), verify=False, ref_n=64, u_hbs=pert)
    assert "hbs_rel_error_vs_oracle" not in leg
