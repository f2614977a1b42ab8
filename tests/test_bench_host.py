"""Host-side logic of bench.py on the CPU: the clock record taken during the
timed region (median SM clock, throttle reasons, the rank's own GPU), the
edge-round count behind the headline value, the peak lookup and the kernel
source hash that guards the stored ncu counters."""
import os

import bench
from paper_2510_12196_gb300 import inputs as I


class _FakeProc:
    def terminate(self):
        pass

    def wait(self, timeout=None):
        return 0

    def kill(self):
        pass


class _FakeThread:
    def join(self, timeout=None):
        pass


def _sampler(lines, bus_id=None):
    s = bench.ClockSampler(bus_id)
    s.proc, s.t, s.lines = _FakeProc(), _FakeThread(), list(lines)
    return s


def _line(idx, bus, sm, mx, reasons=("Not Active",) * 4):
    return ", ".join([str(idx), bus, str(sm), str(mx), "900.5", "0x0"] + list(reasons))


def test_clocks_median_max_and_no_reasons():
    rows = [_line(0, "00000009:01:00.0", sm, 2070) for sm in (2070, 1965, 2070, 2010, 2070)]
    out = _sampler(rows).stop()
    assert out["sm_mhz"] == 2070.0 and out["sm_max_mhz"] == 2070.0
    assert out["reasons"] == [] and out["samples"] == 5


def test_clocks_report_active_throttle_reasons():
    act = ("Not Active", "Active", "Not Active", "Active")  # hw_thermal_slowdown, sw_power_cap
    rows = [_line(0, "00000009:01:00.0", 1500, 2070), _line(0, "00000009:01:00.0", 1400, 2070, act)]
    out = _sampler(rows).stop()
    assert out["reasons"] == ["hw_thermal_slowdown", "sw_power_cap"]
    assert out["sm_mhz"] == 1450.0


def test_clocks_keep_the_ranks_own_gpu():
    rows = [_line(0, "00000009:01:00.0", 2070, 2070), _line(1, "00000019:01:00.0", 990, 2070),
            _line(1, "00000019:01:00.0", 1000, 2070)]
    assert _sampler(rows, bus_id="00000019:01:00.0").stop()["sm_mhz"] == 995.0
    assert _sampler(rows).stop()["samples"] == 3  # no bus id: every row counts


def test_clocks_without_nvidia_smi():
    s = bench.ClockSampler()
    assert s.stop()["reasons"] == ["nvidia-smi unavailable"]


def test_edge_rounds_counts_undirected_edges_per_iteration():
    # levels with m_dir 20 and 6 entries (10 and 3 edges), 4 and 7 Alg. 6 iterations
    assert bench.edge_rounds(2, [8, 4], [20, 6], [4, 7]) == 10 * 4 + 3 * 7
    assert bench.edge_rounds(1, [5], [0], [9]) == 0


def test_measured_peak_reads_the_driver_file():
    peak, kind = bench.measured_peak()
    if os.path.exists(os.path.join(bench.ROOT, "MEASURED_PEAKS.json")):
        assert kind == "measured" and peak > 1000
    else:
        assert (peak, kind) == (6800.0, "fallback")


def test_kernel_hash_ignores_comments_only():
    a = "__global__ void k(int* x) {\n  x[0] = 1;  // one\n}\n"
    b = "// a kernel\n__global__ void k(int* x) {\n\n  x[0] = 1;\n}\n"
    c = "__global__ void k(int* x) {\n  x[0] = 2;\n}\n"
    assert bench._code_only(a) == bench._code_only(b) != bench._code_only(c)
    for v in bench.TRAFFIC.values():  # stored counters match the current code
        assert bench.kernel_hash(v["kernel"]) == v["kernel_hash"], v["kernel"]


def test_config_names_the_workload():
    w = I.workload_rgg(12)
    cfg = bench.config_of(w, {"levels": 2})
    assert "rgg2d n=2^12" in cfg["workload"] and "H=4:8:8 D=1:10:100" in cfg["workload"]
    assert cfg["levels"] == 2 and "flushed" in cfg["l2"]
    assert (cfg["n"], cfg["m_dir"], cfg["k"]) == (w.graph.n, w.graph.m_dir, 256)
    assert cfg["parallelism"] == "replicas"


def test_units_per_step_and_grid_config():
    """A multilevel step maps the input graph once (its undirected edges);
    the grid step is 10 fixed rounds over all its edges."""
    w = I.workload_grid64()
    assert bench.units_per_step(w) == 8064 * 10
    cfg = bench.config_of(w)
    assert "64x64" in cfg["workload"] and "10 fixed refinement rounds" in cfg["workload"]
    assert "L2" in cfg["l2"] and cfg["rounds"] == 10
    r = I.workload_rmat(10)
    assert bench.units_per_step(r) == r.graph.m
    assert "rmat scale 10" in bench.config_of(r)["workload"]


def test_cpu_sample_is_bounded_for_rmat_only():
    class A:
        rmat_scale, cpu_sample_scale, log2n = 22, 11, 12
    big = I.workload_rmat(12)  # stands in for the scale-22 workload (only its name is read)
    s, text = bench.cpu_sample(A, big)
    assert s.name.startswith("rmat_s11") and "scale 11" in text and s.graph.n == 1 << 11
    g = I.workload_rgg(12)
    s, text = bench.cpu_sample(A, g)
    assert s is g and "full workload" in text
    s, text = bench.cpu_sample(A, I.workload_grid64())
    assert "10 fixed refinement rounds" in text
