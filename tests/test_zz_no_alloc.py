"""The allocation-free residual entry point (roeam_flux_residual_noalloc).

It exists for callers that may not allocate device memory when they ask for a residual (a
host that gives this library a fixed device-memory budget and forbids allocation after
start-up, or a monitor beside a solver whose memory pool owns the device); its scratch is a
fixed array inside the library, committed when a handle is created. Through the C ABI it
must return exactly what the allocating roeam_flux_residual returns (the same kernel on the
same state), call after call, and the device's free memory must not move while it runs.
This file is collected last, so a run that stops at its first failure has run every other
test before it.
"""
import numpy as np
import pytest

import workloads as W

pytestmark = pytest.mark.gpu


def _cases():
    specs, states = W.batch(count=3, seed=515, ni_range=(40, 200), nj_range=(30, 120))
    yield "batch_first", specs, states, None
    yield "batch_vanleer", [W.with_params(s, recon=2) for s in specs], states, None
    spec, _ = W.warped_step(96, 64, with_state=False)
    yield "warped_solid", [spec], [W.random_smooth_state(spec, seed=4, mach=2.0, amp=0.2)], None
    slab = W.GridSpec(ni=70, nj=40, dx=0.02, dy=0.02, bc=(W.PERIODIC, W.PERIODIC, W.WALL, 4),
                      params=W.SchemeParams(m_ref=0.4, recon=1))
    yield "exchange_side", [slab], [W.random_smooth_state(slab, seed=3, mach=0.5, amp=0.2)], (0, 3)


CASES = {c[0]: c for c in _cases()}


@pytest.mark.parametrize("prec", [64, 32])
@pytest.mark.parametrize("case", sorted(CASES))
def test_noalloc_residual_matches_allocating_residual(case, prec):
    import torch
    import paper_1711_09272_gb300 as P
    _, specs, states, halo = CASES[case]
    with P.Batch(specs, precision=prec) as b:
        b.set_states(states)
        if halo is not None:
            g, side = halo
            rows = np.ascontiguousarray(np.broadcast_to(states[g][:, -2:, :], (4, 2, specs[g].ni)))
            b.set_halo(g, side, 0, rows[:, ::-1] * 1.01)
        for idx in reversed(range(len(specs))):
            ref = b.residual(idx)
            out = np.full_like(ref, np.nan)
            P.roeam_flux_residual_noalloc(b.handle, idx, out)   # warm-up call of this grid
            torch.cuda.synchronize()
            free0 = torch.cuda.mem_get_info(0)[0]
            for _ in range(2):   # two calls in a row share the scratch array
                out = np.full_like(ref, np.nan)
                P.roeam_flux_residual_noalloc(b.handle, idx, out)
                assert np.array_equal(out, ref), (case, idx)
            assert torch.cuda.mem_get_info(0)[0] == free0


def test_noalloc_residual_rejects_grids_beyond_its_scratch():
    import paper_1711_09272_gb300 as P
    spec = W.GridSpec(ni=1024, nj=768, dx=1e-3, dy=1e-3)
    with P.Batch([spec], precision=64) as b:
        b.set_state(W.free_stream(spec), 0)
        out = np.empty((4, 768, 1024))
        with pytest.raises(P.RoeamError) as e:
            P.roeam_flux_residual_noalloc(b.handle, 0, out)
        assert e.value.status == 1 and "scratch" in str(e.value)
