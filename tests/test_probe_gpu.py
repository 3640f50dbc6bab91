"""The FP64 FMA throughput probe (cpl_probe_fp64), the measured denominator
of the plain path's roofline: its FLOP count follows the documented formula,
it writes nothing, and the rate it measures lies near the FP64 pipe's
nominal rate (2 FMA per clock per SM x 152 SMs) at the clock it ran at --
far above it would mean the sums were optimised away."""
import pytest

from paper_2602_15605_gb300 import coupling

pytestmark = pytest.mark.gpu


def test_probe_counts_and_rate():
    import torch
    from paper_2602_15605_gb300 import build_ext
    build_ext.build()
    sink = torch.zeros(1, dtype=torch.float64, device="cuda")
    n_blocks, iters = 152 * 4, 100
    for _ in range(2):
        flop = coupling.probe_fp64(n_blocks, iters, sink)
    assert flop == 2.0 * 1024 * iters * 256 * n_blocks
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    a.record()
    coupling.probe_fp64(n_blocks, iters, sink)
    b.record()
    torch.cuda.synchronize()
    tflops = flop / (a.elapsed_time(b) * 1e-3) / 1e12
    nominal_at_max = 2.0 * 2 * 152 * 2.07e9 / 1e12
    assert 0.2 * nominal_at_max < tflops < 1.2 * nominal_at_max, tflops
    assert float(sink[0]) == 0.0
