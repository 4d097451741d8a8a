"""The throughput probes behind the measured roofline peaks: each launch does
the work it claims (it lasts the calibrated ~20 ms, so no chain was folded
away by the compiler), and the FMA rates sit near the unit counts of the
GPU's SMs at its maximum clock (128 FP32 and 2 FP64 FMA lanes per SM per
clock)."""
import pytest

pytestmark = pytest.mark.gpu


def test_probes_measure_real_work():
    import torch
    assert torch.cuda.is_available(), "GPU tests need CUDA"
    from paper_1503_03806_gb300 import build
    build.build()
    from paper_1503_03806_gb300 import helk
    ctx = helk.Context(0)
    try:
        nsm = torch.cuda.get_device_properties(0).multi_processor_count
        max_ghz = 2.07  # the highest SM clock of the part; the probe cannot beat it
        rates = {}
        for kind in (helk.HELK_PROBE_FFMA, helk.HELK_PROBE_DFMA, helk.HELK_PROBE_MUFU_RCP,
                     helk.HELK_PROBE_MUFU_EX2):
            ops, ms = ctx.peak_probe(kind)
            assert ms >= 5.0, (kind, ms)
            rates[kind] = ops
        ffma_unit = 128 * 2 * nsm * max_ghz * 1e9
        dfma_unit = 2 * 2 * nsm * max_ghz * 1e9
        assert 0.5 * ffma_unit <= rates[helk.HELK_PROBE_FFMA] <= 1.02 * ffma_unit
        assert 0.5 * dfma_unit <= rates[helk.HELK_PROBE_DFMA] <= 1.02 * dfma_unit
        # MUFU: at least 8 results per clock per SM, far below the FMA rate
        for kind in (helk.HELK_PROBE_MUFU_RCP, helk.HELK_PROBE_MUFU_EX2):
            assert 8 * nsm * 1.0e9 <= rates[kind] <= 0.5 * ffma_unit / 2, (kind, rates[kind])
        with pytest.raises(helk.HelkError):
            ctx.peak_probe(7)
    finally:
        ctx.close()
