"""The throughput probe behind the roofline denominators (phia_mma_peak): tcgen05 e4m3
and bf16 MMAs and the warp-level int8 mma.sync route give positive rates, e4m3 above
bf16 (twice the operand rate per instruction), and invalid arguments are refused."""
import pytest

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


def test_probe_rates(gpu_lib):
    phia = gpu_lib
    rates = {}
    for name, op in (("e4m3", phia.OP_E4M3), ("bf16", phia.OP_BF16), ("s8", phia.PEAK_S8_MMA_SYNC)):
        ms, tf = phia.mma_peak(op, 256, 2000)
        assert ms > 0 and tf > 0, name
        rates[name] = tf
    assert rates["e4m3"] > 1.5 * rates["bf16"]
    with pytest.raises(phia.PhiaError) as ei:
        phia.mma_peak(7, 256, 10)
    assert ei.value.code == phia.EINVAL
    with pytest.raises(phia.PhiaError) as ei:
        phia.mma_peak(phia.OP_E4M3, 24, 10)
    assert ei.value.code == phia.EINVAL
