"""The library's device self-test: the integer-arithmetic binary32 <-> binary64
conversions used by the FP64 refinement kernels agree bit for bit with the
hardware conversions (IEEE 754 round to nearest, ties to even; exact widening
with a power-of-two scale)."""
import pytest

from gpu_util import require_gpu

pytestmark = pytest.mark.gpu


def test_conversions_match_hardware():
    require_gpu()
    from paper_1307_2036_gb300 import ellsolve
    assert ellsolve.selftest(1 << 26) == 0
