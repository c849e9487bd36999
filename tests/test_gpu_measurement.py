"""Measurement aids: the FP32 rate probe behind the bench's measured FP32 peak."""
import pytest

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def fq():
    import torch
    assert torch.cuda.is_available()
    import paper_1508_07621_gb300 as fq
    return fq


@pytest.mark.parametrize("packed", [True, False])
def test_fp32_probe_does_the_work_it_counts(fq, packed):
    """Three CTAs (a 1000-float buffer holds 3 x 256 sums): the flop count is 32 per thread and
    iteration, and every thread's 16 chains x = 0.999 x + 0.001 have converged to 1 (sum 16)."""
    import torch
    out = torch.full((1000,), float("nan"), dtype=torch.float32, device="cuda")
    iters = 16384
    flops = fq.floquet_probe_fp32(packed, iters, out)
    torch.cuda.synchronize()
    assert flops == 3 * 256 * iters * 32
    assert torch.allclose(out[:768], torch.full((768,), 16.0, device="cuda"), atol=1e-3)
    assert torch.isnan(out[768:]).all()


def test_fp32_probe_rejects_a_short_buffer(fq):
    import torch
    with pytest.raises(fq.FloquetError):
        fq.floquet_probe_fp32(True, 10, torch.empty(100, dtype=torch.float32, device="cuda"))
