"""aes_measure_peaks: the device rates the benchmark's roofline divides by.

The per-SM rates are measured with clock64 on each SM, so they are counts
per clock that the architecture fixes: one 128-byte shared-memory wavefront
(32 conflict-free 32-bit loads), 64 lanes of three-input logic or byte
permutes and 128 lanes of 32-bit adds per clock per SM.  The link figures
are bandwidths and only need to be plausible for NVLink-C2C."""
import pytest

pytestmark = pytest.mark.gpu


def test_measured_rates_are_the_architectures(cuda, aes):
    r = aes.measure_peaks()
    assert r["sms"] == cuda.cuda.get_device_properties(0).multi_processor_count
    assert 30.0 <= r["lds32_per_clk_sm"] <= 32.5, r
    assert 60.0 <= r["lop3_per_clk_sm"] <= 64.5, r
    assert 60.0 <= r["prmt_per_clk_sm"] <= 64.5, r
    assert 120.0 <= r["iadd_per_clk_sm"] <= 128.5, r
    assert 500.0 <= r["sm_mhz_during_probe"] <= 2200.0, r
    for k in ("h2d_gbs", "d2h_gbs", "h2d_d2h_each_way_gbs", "zero_copy_each_way_gbs"):
        assert 20.0 <= r[k] <= 1000.0, (k, r)


def test_measure_peaks_refuses_a_null_output(aes):
    assert aes.lib().aes_measure_peaks(None) == aes.AES_EINVAL
