"""Host logic of bench.py that feeds its JSON line: the DRAM-traffic lookup
(keyed by kernel, storage, multi-step shape and the kernel's sources) and
the FP32-pipe figure's operation count."""
import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)
import bench  # noqa: E402


def _lines():
    path = os.path.join(ROOT, "profiles", "dram_traffic.txt")
    out = []
    for line in open(path):
        f = line.split()
        if f and not f[0].startswith("#"):
            out.append(f)
    return out


def test_every_traffic_line_matches_its_kernel_sources():
    """A committed line is only used while its kernel's sources are those it
    was captured on: every line names a known kernel and the current hash."""
    lines = _lines()
    assert lines
    for f in lines:
        kern = f[0].split(":")[0]
        assert kern in bench.KERNEL_SOURCES, f[0]
        assert f[5] == bench.kernel_source_hash(kern), f[0]


def test_traffic_lookup_scales_and_keys_by_shape():
    lines = {(f[0], f[1]): f for f in _lines()}
    f = lines[("step_wave:5x128", "fp32")]
    full = float(f[4])
    got = bench.ncu_traffic("step_wave", "fp32", 8192, 8192, {"steps": 5, "rows": 128})
    assert got == pytest.approx(full)
    # traffic grows with the sites: half the rows, half the bytes
    half = bench.ncu_traffic("step_wave", "fp32", 8192, 4096, {"steps": 5, "rows": 128})
    assert half == pytest.approx(full / 2)
    # a shape without a capture, another storage, or no shape for a
    # multi-step kernel: no traffic figure rather than a wrong one
    assert bench.ncu_traffic("step_wave", "fp32", 8192, 8192, {"steps": 3, "rows": 64}) is None
    assert bench.ncu_traffic("step_wave", "bf16", 8192, 8192, {"steps": 5, "rows": 128}) is None
    assert bench.ncu_traffic("step_wave", "fp32", 8192, 8192) is None
    # single-step kernels are keyed by name alone
    v = lines[("step_vector", "fp32")]
    assert bench.ncu_traffic("step_vector", "fp32", 8192, 8192) == pytest.approx(float(v[4]))
    assert bench.ncu_traffic("no_such_kernel", "fp32", 8192, 8192) is None


def test_fp32_operation_count_of_the_collision():
    """48 operations per node: 15 for rho, m_x, m_y (7 + 4 + 4 with the
    shared d_4 - d_6 and d_7 - d_5), 9 for the flux terms ((1 - zeta) m:
    2, -rho: 1, t_a, t_b: 2, t_p, t_m: 2 + 2), 3 per population."""
    assert 7 + 4 + 4 + (2 + 1 + 2 + 4) + 3 * 8 == 48
    for precision in ("fp32", "fp16", "bf16"):
        assert bench.FP32_OPS_PER_UPDATE[precision] == 48
    assert "fp64" not in bench.FP32_OPS_PER_UPDATE
