"""The library's own device-memory high-water mark (hh_stats_t.mem_peak_bytes):
positive after a prediction, below the device's memory, and growing with N."""
import pytest

import hh_synth

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")
import paper_2505_08174_b300 as hh  # noqa: E402


def test_peak_memory_is_reported():
    import gc
    gc.collect()                      # structures of earlier tests are freed before the marks are taken
    torch.cuda.synchronize()
    c = hh.Context()
    c.set_mlp(hh_synth.mlp_params(32, 7), 32)
    total = torch.cuda.get_device_properties(0).total_memory
    peaks = []
    for n in (2000, 40000):
        X = torch.as_tensor(hh_synth.rsa_cube(n, 0.1, seed=n)).cuda()
        c.predict(X, X.clone(), hh.Params(precision="bf16", leaf_size=64))
        m = c.stats()["mem_peak_bytes"]
        assert 0 < m < total
        peaks.append(m)
    assert peaks[1] > peaks[0]
