"""The FP64 FMA probe that sets the measured peak of the roofline: it runs, and its
rate is physically plausible (between a third of and just above the FP64 rate
the SM count and the maximum SM clock allow, 2 DFMA lanes per clock per SM)."""
import json
import os

import pytest

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_fp64_probe_rate_is_plausible():
    import torch

    import paper_1606_05836_gb300 as pg
    from paper_1606_05836_gb300 import build
    build.build()
    dev = torch.device("cuda", 0)
    sms = torch.cuda.get_device_properties(dev).multi_processor_count
    mhz = 2070.0
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            mhz = float(json.load(f).get("sm_max_mhz", mhz))
    except (OSError, ValueError):
        pass
    pg.fp64_fma_probe(64, 4 * sms, 256, dev)
    torch.cuda.synchronize(dev)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    fmas = pg.fp64_fma_probe(1 << 14, 4 * sms, 256, dev)
    e1.record()
    torch.cuda.synchronize(dev)
    rate = fmas / (e0.elapsed_time(e1) / 1e3)
    ceiling = sms * 2 * mhz * 1e6
    print("\nFP64 probe: %.3g DFMA/s = %.3f of %d SMs x 2 x %.0f MHz" % (rate, rate / ceiling, sms, mhz))
    assert 0.33 * ceiling < rate < 1.05 * ceiling
