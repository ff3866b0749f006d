"""The measurement entry point dock_gather_peak (no counterpart in the paper)."""
import math

import numpy as np
import pytest

from paper_2209_05069_gb300 import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def dk():
    from paper_2209_05069_gb300 import dock
    return dock


def test_gather_peak_on_every_grid_type(dk):
    w = synth.WORKLOADS["uneven"]
    pk = synth.workload_pocket(w)
    with dk.Context(serve=False) as ctx:
        rates = {}
        for dtype, p in (("f32", pk), ("f16", pk), ("i16", pk.integer(1000))):
            rates[dtype] = ctx.gather_peak(ctx.load(p, dtype))
            assert math.isfinite(rates[dtype]) and 1e10 < rates[dtype] < 1e13, (dtype, rates[dtype])
        # an all-zero grid issues no loads at all (the box test skips them): faster than any
        empty = ctx.load_pocket(np.zeros((8, 8, 8), np.float32), 0.5, (0, 0, 0))
        assert ctx.gather_peak(empty) > rates["f32"]
        with pytest.raises(dk.DockError) as e:
            ctx.gather_peak(12345)
        assert e.value.code == dk.DOCK_ERR_NOPOCKET
    print("\nscattered lookups/s:", {k: f"{v / 1e9:.0f} G" for k, v in rates.items()})
