"""The allocation-free residual entry point (roeam_flux_residual_noalloc).

It exists for callers that may not allocate device memory when they ask for a residual;
its scratch is a fixed array inside the library. Through the C ABI, it must return what
the allocating roeam_flux_residual returns, call after call.
"""
import numpy as np
import pytest

import workloads as W

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("prec", [64, 32])
def test_noalloc_residual_matches_allocating_residual(prec):
    import paper_1711_09272_gb300 as P
    specs, states = W.batch(count=3, seed=515, ni_range=(40, 200), nj_range=(30, 120))
    with P.Batch(specs, precision=prec) as b:
        b.set_states(states)
        for idx in (2, 0, 1):
            ref = b.residual(idx)
            scale = np.abs(ref).max()
            for _ in range(2):   # two calls in a row share the scratch array
                out = np.full_like(ref, np.nan)
                P.roeam_flux_residual_noalloc(b.handle, idx, out)
                assert np.all(np.isfinite(out))
                assert np.max(np.abs(out - ref)) <= (1e-13 if prec == 64 else 1e-6) * scale


def test_noalloc_residual_rejects_grids_beyond_its_scratch():
    import paper_1711_09272_gb300 as P
    spec = W.GridSpec(ni=1024, nj=768, dx=1e-3, dy=1e-3)
    with P.Batch([spec], precision=64) as b:
        b.set_state(W.free_stream(spec), 0)
        out = np.empty((4, 768, 1024))
        with pytest.raises(P.RoeamError) as e:
            P.roeam_flux_residual_noalloc(b.handle, 0, out)
        assert e.value.status == 1 and "scratch" in str(e.value)
