"""The measured-peak diagnostic (slqr_measure_peak) on the GPU: the FP64 FMA
probe and the TF32 tensor-core probe run, leave the status word clean, and
give rates of the right order for a GB300 (the FP64 pipe's derived peak is
4 flop per clock per SM, 1.26 TFLOP/s at 2070 MHz on 152 SMs; the TF32 dense
tensor rate is of the order of a PFLOP/s)."""
import pytest

pytestmark = pytest.mark.gpu


def test_peak_probes():
    from paper_2506_09463_gb300 import abi, api
    with api.Context(0) as ctx:
        st, fp64 = abi.slqr_measure_peak(ctx.ctx, abi.SLQR_PEAK_FP64_FMA)
        assert st == abi.SLQR_OK, abi.slqr_last_error(ctx.ctx)
        st, tf32 = abi.slqr_measure_peak(ctx.ctx, abi.SLQR_PEAK_TF32_TC)
        assert st == abi.SLQR_OK, abi.slqr_last_error(ctx.ctx)
        assert ctx.sync() == 0
        assert 0.5 < fp64 < 2.0, fp64
        assert 100.0 < tf32 < 3000.0, tf32
        assert abi.slqr_measure_peak(ctx.ctx, 7)[0] == abi.SLQR_EINVAL
