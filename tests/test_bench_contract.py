"""Host-side pieces of bench.py that the JSON line depends on: the algorithmic
bytes behind the roofline fractions, the ncu traffic table, and the parsing of
the nvidia-smi clock samples.  No GPU needed."""
import bench
from paper_2009_04619_gb300 import synth


def test_algorithmic_bytes_per_launch_512():
    """512^3 computed, 448^3 inner: N = 134,217,728 points, P = 44,302,336 PML
    points.  fp32: 16 N + 8 P; 16-bit wavefields: 10 N + 8 P; 16-bit difference
    form (u^n, d^n read, u^{n+1}, d^{n+1} written): 12 N + 8 P."""
    w = synth.LARGE
    assert (w.points, w.points - w.nx * w.ny * w.nz) == (134_217_728, 44_302_336)
    assert bench._alg_bytes_per_launch(w) == 2_501_902_336
    assert bench._alg_bytes_per_launch(w, wave_bytes=2) == 1_696_595_968
    assert bench._alg_bytes_per_launch(w, wave_bytes=2, wave_fields=4) == 1_965_031_424


def test_gradient_bytes_per_shot():
    """256^3 computed, 224^3 inner (N = 16,777,216, P = 5,537,792), 2000 steps,
    checkpoints every 100 (20 segments, each saved and restored: 2 x 24 B/pt) and
    63 folds of 24 B/pt: 2000 (64 N + 24 P) + (960 + 1512) N."""
    w = synth.GRADIENT
    N, P = w.points, w.points - w.nx * w.ny * w.nz
    assert (N, P) == (16_777_216, 5_537_792)
    assert bench._gradient_alg_bytes(w, 2000, 100) == 2_454_770_941_952


def test_traffic_table_is_plausible():
    """Every ncu traffic figure of the 512^3 step lies between the algorithmic
    bytes and 1.2 times them, and the source hash is stable."""
    alg = bench._alg_bytes_per_launch(synth.LARGE)
    assert bench.NCU_TRAFFIC
    for key, traffic in bench.NCU_TRAFFIC.items():
        assert len(key) == 16 and alg <= traffic <= 1.2 * alg, (key, traffic)
    assert bench._kernel_hash() == bench._kernel_hash()


class _FakeSmi:
    def __init__(self, text):
        self.text = text

    def terminate(self):
        pass

    def communicate(self, timeout=None):
        return self.text, ""


def test_clock_samples_parsed():
    """Median SM clock, the largest max clock, and every throttle reason that was
    Active in some sample (malformed lines skipped)."""
    lines = [
        "0, 2070, 2070, 910.5, 0x0, Not Active, Not Active, Not Active, Not Active",
        "0, 2040, 2070, 1390.0, 0x4, Not Active, Not Active, Not Active, Active",
        "0, 2070, 2070, 1200.0, 0x0, Not Active, Not Active, Not Active, Not Active",
        "garbage",
    ]
    s = bench.ClockSampler("GPU-0")
    s.proc = _FakeSmi("\n".join(lines))
    out = s.stop()
    assert out["sm_mhz"] == 2070.0 and out["sm_max_mhz"] == 2070.0 and out["samples"] == 3
    assert out["reasons"] == ["sw_power_cap"]
    s.proc = _FakeSmi("0, 1500, 2070, 800, 0x8, Active, Not Active, Active, Not Active\n")
    out = s.stop()
    assert out["reasons"] == ["hw_slowdown", "sw_thermal_slowdown"]
    s.proc = None
    assert s.stop()["sm_mhz"] is None
