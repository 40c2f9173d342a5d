"""coot_probe_device: the device's arithmetic and memory rates from small
kernels timed with CUDA events (the denominators of the FP64 trees' and the
end-to-end figure's rooflines).  The rates must be positive and ordered as
the hardware orders them."""
import pytest
import torch

from paper_2508_11385_gb300 import lib as L

pytestmark = pytest.mark.gpu


def test_probe_rates_are_plausible():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    r = L.coot_probe_device(torch.cuda.current_device())
    for k in ("f32_add", "f32_fma", "f32_div", "f32_exp", "f64_add", "f64_fma", "f64_div", "f64_exp", "read_gbs",
              "copy_gbs", "host_read_gbs", "host_write_gbs"):
        assert r[k] > 0, k
    assert r["f32_add"] > 8 * r["f64_add"]       # FP64 runs far below FP32 on this part
    assert r["f32_fma"] > r["f32_exp"] > 0 and r["f64_fma"] > r["f64_div"]
    assert r["read_gbs"] > 10 * r["host_read_gbs"]  # HBM against the host link
    props = torch.cuda.get_device_properties(torch.cuda.current_device())
    assert r["sms"] == props.multi_processor_count and r["l2_bytes"] == props.L2_cache_size
    assert r["buffer_bytes"] >= 8 * r["l2_bytes"]
