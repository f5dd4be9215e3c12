"""wd_norm2_noalloc: the norm for callers that cannot allocate device memory.

Such callers (plug-ins whose host framework owns all device memory and
forbids raw cudaMalloc, latency-critical loops that cannot afford cudaMalloc's
implicit synchronisation) cannot create a context, whose scratch is allocated.  The entry point keeps its
scratch in a fixed array inside the library.  This test calls it through the C
ABI twice in a row and checks each result against wd_norm2's, and checks that a
field too large for the fixed scratch is refused.  It lives in a file that
pytest collects last, and passes alone in a fresh process or after the rest.
"""
import numpy as np
import pytest

import paper_1901_07294_gb300 as wd
import synth
from tests._gpu import pack_field

pytestmark = pytest.mark.gpu

RTOL = 1e-12   # the two entry points differ only in the FP64 summation order


@pytest.mark.parametrize("prec", [wd.F64, wd.F32, wd.F16, wd.BF16, wd.DF])
@pytest.mark.parametrize("dims,sites", [((8, 8, 8, 8), wd.SITES_FULL), ((4, 6, 8, 10), wd.SITES_EVEN),
                                        ((32, 32, 32, 32), wd.SITES_FULL)])
def test_noalloc_norm_matches_context_norm_twice(prec, dims, sites):
    import torch
    ctx = wd.Context(0)
    x = pack_field(ctx, dims, sites, prec, synth.spinor(dims, seed=4242))
    ref = torch.zeros(1, dtype=torch.float64, device="cuda")
    wd.norm2(ctx, dims, sites, prec, x, ref)
    got = torch.full((2,), -1.0, dtype=torch.float64, device="cuda")
    wd.norm2_noalloc(dims, sites, prec, x, got[0:1])
    wd.norm2_noalloc(dims, sites, prec, x, got[1:2])
    torch.cuda.synchronize()
    r = ref.item()
    assert r > 0
    for k in range(2):
        assert abs(got[k].item() - r) / r < RTOL, (k, got[k].item(), r)


def test_noalloc_refuses_fields_beyond_the_fixed_scratch():
    import torch
    x = torch.zeros(16, dtype=torch.uint8, device="cuda")
    out = torch.zeros(1, dtype=torch.float64, device="cuda")
    # 64^3 x 16 full field = 4,194,304 sites > 2,097,152; refused before any launch
    with pytest.raises(wd.WdError) as e:
        wd.norm2_noalloc((64, 64, 64, 16), wd.SITES_FULL, wd.F32, x, out)
    assert e.value.status == wd.WD_EINVAL
    assert "fixed scratch" in str(e.value)
