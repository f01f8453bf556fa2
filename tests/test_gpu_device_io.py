"""Device-pointer state I/O (roeam_set_state_device / roeam_get_state_device): a caller whose
state already lives on the GPU (here a PyTorch float64 tensor) steps through the C ABI without
a host round trip, and gets exactly what the host-array calls give."""
import numpy as np
import pytest

import workloads as W

pytestmark = pytest.mark.gpu


def P():
    import paper_1711_09272_gb300 as pkg
    return pkg


@pytest.mark.parametrize("recon", [0, 2])
@pytest.mark.parametrize("prec", [64, 32])
def test_device_io_matches_host_path(prec, recon):
    import torch
    specs, states = W.batch(count=7, seed=33, ni_range=(20, 150), nj_range=(10, 90), recon=recon)
    packed = np.concatenate([U.ravel() for U in states])
    with P().Batch(specs, precision=prec) as b:
        b.set_states(states)
        b.step(0.5, nsteps=3)
        ref = b.get_states()
        ref_dt = b.step(0.5, nsteps=1, want_dt=True)
        ref1 = b.get_states()
    dev = torch.from_numpy(packed).cuda()
    out = torch.full_like(dev, float("nan"))
    with P().Batch(specs, precision=prec) as b:
        b.set_state_device(dev, -1)
        b.step(0.5, nsteps=3)
        b.get_state_device(out, -1)
        torch.cuda.synchronize()
        got = out.cpu().numpy()
        dt = b.step(0.5, nsteps=1, want_dt=True)
        # one grid at a time, on a caller stream that is not the handle's
        s = torch.cuda.Stream()
        with torch.cuda.stream(s):
            outs = [torch.empty(4 * sp.ni * sp.nj, dtype=torch.float64, device="cuda") for sp in specs]
            for k in range(len(specs)):
                b.get_state_device(outs[k], k, stream=s.cuda_stream)
            sums = [o.sum() for o in outs]   # ordered after the library's copies on s
        s.synchronize()
        got1 = [o.cpu().numpy().reshape(4, sp.nj, sp.ni) for o, sp in zip(outs, specs)]
    off = 0
    for k, sp in enumerate(specs):
        n = 4 * sp.ni * sp.nj
        assert np.array_equal(got[off:off + n].reshape(4, sp.nj, sp.ni), ref[k]), k
        assert np.array_equal(got1[k], ref1[k]), k
        assert float(sums[k]) == pytest.approx(float(ref1[k].sum()), rel=1e-12)
        off += n
    assert np.array_equal(dt, ref_dt)


def test_device_io_set_one_grid_and_ordering():
    """Setting one grid from a tensor written on another stream, then stepping, equals the host
    path; the call is ordered after the caller's stream without a host wait."""
    import torch
    spec = W.GridSpec(ni=130, nj=70, dx=0.01, dy=0.01, params=W.SchemeParams(m_ref=0.5))
    U = W.random_rough_state(spec, seed=4, mach=0.8, jump=0.3)
    with P().Batch([spec, spec], precision=32) as b:
        b.set_states([U, U])
        b.step(0.5, nsteps=2)
        ref = b.get_states()
    s = torch.cuda.Stream()
    with P().Batch([spec, spec], precision=32) as b:
        b.set_states([np.ones_like(U), U])
        with torch.cuda.stream(s):
            src = torch.zeros(U.size, dtype=torch.float64, device="cuda")
            torch.cuda._sleep(2_000_000)            # the copy below lands late on s
            src.copy_(torch.from_numpy(U.ravel()).cuda(non_blocking=False))
            b.set_state_device(src, 0, stream=s.cuda_stream)
        b.step(0.5, nsteps=2)
        got = b.get_states()
    assert np.array_equal(got[0], ref[0]) and np.array_equal(got[1], ref[1])


def test_device_io_rejects_host_memory():
    import torch
    spec = W.GridSpec(ni=16, nj=8, dx=0.1, dy=0.1)
    with P().Batch([spec], precision=64) as b:
        host = torch.zeros(4 * 16 * 8, dtype=torch.float64)
        with pytest.raises(P().RoeamError) as e:
            b.set_state_device(host, 0)
        assert e.value.status == 1
        with pytest.raises(P().RoeamError):
            b.get_state_device(host, 0)


@pytest.mark.parametrize("prec", [32, 64])
def test_single_precision_host_arrays(prec):
    """roeam_set_state_f32 / roeam_get_state_f32 / roeam_step_host_f32: float32 host arrays give
    the state the float64 calls give for the same (float32-representable) input, bit for bit
    after rounding the float64 output to float32; an FP32 handle loses nothing either way."""
    import torch
    specs, states = W.batch(count=30, seed=91, ni_range=(20, 150), nj_range=(10, 90))
    packed32 = np.concatenate([U.ravel() for U in states]).astype(np.float32)
    packed64 = packed32.astype(np.float64)
    with P().Batch(specs, precision=prec) as b:
        b.set_state(packed64, -1)
        dt_ref = b.step(0.5, nsteps=3, want_dt=True)
        ref = np.concatenate([u.ravel() for u in b.get_states()])
    with P().Batch(specs, precision=prec) as b:
        P().roeam_set_state_f32(b.handle, -1, packed32)
        out = np.empty_like(packed32)
        P().roeam_get_state_f32(b.handle, -1, out)
        assert np.array_equal(out, packed32)
        b.step(0.5, nsteps=3)
        P().roeam_get_state_f32(b.handle, -1, out)
        assert np.array_equal(out, ref.astype(np.float32))
    h_in = torch.from_numpy(packed32.copy()).pin_memory()
    h_out = torch.empty_like(h_in).pin_memory()
    dt = np.zeros(len(specs))
    with P().Batch(specs, precision=prec) as b:
        P().roeam_step_host_f32(b.handle, 0.5, 0.0, 3, h_in, h_out, dt)
        got = h_out.numpy().copy()
        assert np.array_equal(np.concatenate([u.ravel() for u in b.get_states()]).astype(np.float32), got)
    assert np.array_equal(got, ref.astype(np.float32))
    assert np.array_equal(dt, dt_ref)
    if prec == 32:   # an FP32 state read back in float64 is exact
        assert np.array_equal(ref, ref.astype(np.float32).astype(np.float64))
