"""The measured memory ceilings the step kernel's roofline divides by
(sk_peaks.h): positive, ordered as the hardware orders them (random 4-byte
gathers below conflict-free 16-byte loads), and within a plausible factor of
the nominal figures (shared memory 128 bytes per clock per SM; L2 below
shared memory)."""
import pytest

from paper_2102_05613_gb300 import sk

from gpu_util import need_gpu

pytestmark = pytest.mark.gpu


def test_peak_probes_are_plausible():
    torch = need_gpu()
    props = torch.cuda.get_device_properties(0)
    sms = props.multi_processor_count
    vec = sk.peak_smem(sk.SK_PEAK_SMEM_VEC16, iters=256, reps=2)
    gat = sk.peak_smem(sk.SK_PEAK_SMEM_GATHER4, iters=256, reps=2)
    l2 = sk.peak_l2_read(32 << 20, passes=16, reps=2)
    nominal_smem = sms * 128 * 2.1e9 / 1e9  # GB/s at the part's top clock
    assert 0.2 * nominal_smem < vec < 1.05 * nominal_smem, (vec, nominal_smem)
    assert 0.0 < gat < vec
    assert 0.0 < l2 < vec


def test_tensor_probe_is_plausible():
    # the recompute kernel's own MMA loop with nothing else to do: positive,
    # below the part's nominal dense rates (4.5 PFLOP/s FP8, 2.25 PFLOP/s bf16)
    # with room for clocks, and FP8 faster than bf16
    need_gpu()
    f8 = sk.peak_tensor(sk.SK_J_PM1, tiles=32, reps=2)
    b16 = sk.peak_tensor(sk.SK_J_GAUSS, tiles=32, reps=2)
    assert 100.0 < f8 < 4700.0, f8
    assert 50.0 < b16 < 2400.0, b16
    assert f8 > b16
