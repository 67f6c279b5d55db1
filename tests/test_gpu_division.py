"""The uint16 path's division S = L+/(2N), formed from a table of 2N and its
correctly rounded reciprocal with Markstein's correction, equals IEEE float32
division bit for bit for every numerator a uint16 frame's L+ can take and every
table entry (lacos_selftest_division checks all 3.4e10 pairs on the device)."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def lacos():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2602_17938_gb300 import build, lacos as lc
    build.build()
    return lc


def _params():
    # the workloads' gains and read noises, edge values, and a seeded sweep
    fixed = [(1.0, 1.5), (0.8, 1.2), (1.0, 0.0), (3.7, 0.01), (0.05, 25.0), (12.0, 4.0)]
    rng = np.random.default_rng(17)
    sweep = [(float(rng.uniform(0.3, 4.0)), float(rng.uniform(0.0, 12.0))) for _ in range(6)]
    return fixed + sweep


@pytest.mark.parametrize("gain,readnoise", _params())
def test_table_division_is_ieee_division(lacos, gain, readnoise):
    assert lacos.selftest_division(gain, readnoise) == 0


def test_selftest_rejects_bad_arguments(lacos):
    with pytest.raises(lacos.LacosError):
        lacos.selftest_division(0.0, 1.0)
    with pytest.raises(lacos.LacosError):
        lacos.selftest_division(1.0, -1.0)
