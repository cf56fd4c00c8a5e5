"""The bit-level FP64 helpers (csrc/gs_bits.cuh) give, for every input the device self-test draws,
exactly the result of the instruction each replaces: FP64 -> FP32 rounding and FP32 -> FP64
widening (as this library is built, with FP32 flush-to-zero), FP64 comparisons, NaN and finiteness
tests, sign operations; log2 within its stated FP32 accuracy. The FP32-stage kernels rely on this to
keep conversions and comparisons off the FP64 pipe without changing any result."""
import pytest

from gpu_util import ensure_built
from paper_2609_28458_gb300 import api

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("seed", [0, 0x5eed0001, 0xfeedfacecafebeef])
def test_bit_helpers_match_the_instructions(seed):
    ensure_built()
    res = api.selftest(n=1 << 23, seed=seed)
    bad = {k: (cnt, hex(witness)) for k, (cnt, witness) in res.items() if cnt}
    assert not bad, bad
