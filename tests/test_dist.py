"""Host logic of the multi-GPU benchmark with two gloo ranks on the CPU: every rank gets its
own seeded batch (weak scaling, no data-path collective) and the reported time is the
maximum over ranks."""
import os
import socket

import pytest
import torch.multiprocessing as mp


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank, world, port, out):
    import sys
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    sys.path.insert(0, root)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    import torch.distributed as dist
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    import workloads as W
    specs, _ = W.batch(4, seed=bench.rank_seed(rank))
    ms = 10.0 + 5.0 * rank
    cells = sum(s.ncells for s in specs)
    out[rank] = (bench.reduce_max(ms, world, device="cpu"), [s.ni for s in specs], cells,
                 bench.reduce_sum(cells, world, device="cpu"))
    dist.barrier()
    dist.destroy_process_group()


def test_two_rank_weak_scaling_host_logic():
    world = 2
    mgr = mp.Manager()
    out = mgr.dict()
    mp.spawn(_worker, args=(world, _free_port(), out), nprocs=world, join=True)
    t0, ni0, c0, tot0 = out[0]
    t1, ni1, c1, tot1 = out[1]
    assert t0 == t1 == 15.0                 # both ranks report the slowest rank's time
    assert ni0 != ni1                       # independent batches per rank
    assert tot0 == tot1 == c0 + c1          # the whole job's cells, whatever each rank drew
    import bench
    v = bench.weak_value(tot0, 10, t0)
    assert v == pytest.approx((c0 + c1) * 3 * 10 / 15e-3 / 1e9)


# ----------------------------------------------------------------------------- row slabs
def _slab_case(name):
    import workloads as W
    if name == "warped_solid":
        # the Mach-3 step (solid block, walls, inflow, outflow, van Leer) on a small warped grid
        spec, _ = W.warped_step(24, 20, with_state=False)
        return spec, W.random_smooth_state(spec, seed=6, mach=2.0, amp=0.2)
    if name == "periodic":
        spec = W.GridSpec(ni=22, nj=17, dx=0.05, dy=0.06, params=W.SchemeParams(m_ref=0.4, recon=2))
    else:
        spec = W.GridSpec(ni=20, nj=18, dx=0.05, dy=0.05, bc=(W.PERIODIC, W.PERIODIC, W.WALL, W.INFLOW),
                          inflow=(1.1, 0.3, -0.2, 0.9), params=W.SchemeParams(m_ref=0.5, eps1=1))
    U = W.random_smooth_state(W.GridSpec(ni=spec.ni, nj=spec.nj, dx=spec.dx, dy=spec.dy, params=spec.params),
                              seed=4, mach=0.6, amp=0.3)
    return spec, U


def _slab_worker(rank, world, port, name, out):
    import sys
    here = os.path.dirname(os.path.abspath(__file__))
    sys.path.insert(0, os.path.dirname(here))
    sys.path.insert(0, here)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    import numpy as np
    import torch
    import torch.distributed as dist
    dist.init_process_group("gloo", rank=rank, world_size=world)
    from paper_1711_09272_gb300.slab import DistExchange, SlabStepper
    from slab_oracle import OracleSlab
    spec, U = _slab_case(name)
    st = SlabStepper(spec, world, [rank], DistExchange(torch), make_slab=OracleSlab)
    st.set_state(U)
    dts = [st.step(0.5) for _ in range(3)]
    mine = st.get_state(np.zeros_like(U))
    j0, j1 = st.slabs[rank][1]
    out[rank] = (j0, j1, mine[:, j0:j1].copy(), dts)
    dist.barrier()
    dist.destroy_process_group()


@pytest.mark.parametrize("name", ["periodic", "wall_inflow", "warped_solid"])
def test_two_rank_row_slabs_match_the_whole_grid(name):
    """A grid split into two row slabs on two gloo ranks (halo exchange before every stage, a
    max-reduction of the rate per step) advances exactly like the whole grid: the stepper's
    choreography, tags and neighbour maps, with the FP64 oracle standing in for the GPU."""
    import numpy as np
    import oracle
    world = 2
    mgr = mp.Manager()
    out = mgr.dict()
    mp.spawn(_slab_worker, args=(world, _free_port(), name, out), nprocs=world, join=True)
    spec, U = _slab_case(name)
    g = oracle.OracleGrid(spec)
    Ur = U.copy()
    for r in range(world):
        assert out[r][3] == out[0][3]          # one global dt per step on every rank
    for dt in out[0][3]:
        Ur, dto = g.step(Ur, cfl=0.5)
        assert abs(dto - dt) <= 1e-14 * dt
    got = np.zeros_like(U)
    for r in range(world):
        j0, j1, rows, _ = out[r]
        got[:, j0:j1] = rows
    # (the oracle builds Cartesian face vectors from vertex coordinates j dy, so a slab's
    #  local row numbering rounds them differently in the last bit)
    assert np.max(np.abs(got - Ur).reshape(4, -1).max(axis=1) / np.abs(Ur).reshape(4, -1).max(axis=1)) < 1e-13


def test_local_three_slabs_match_the_whole_grid():
    """Three slabs in one process (LocalExchange), periodic in y: each slab's two neighbours."""
    import sys
    sys.path.insert(0, os.path.dirname(os.path.abspath(__file__)))
    import numpy as np
    import oracle
    from paper_1711_09272_gb300.slab import LocalExchange, SlabStepper, slab_rows
    from slab_oracle import OracleSlab
    spec, U = _slab_case("periodic")
    assert slab_rows(17, 3) == [(0, 6), (6, 12), (12, 17)]
    st = SlabStepper(spec, 3, [0, 1, 2], LocalExchange(), make_slab=OracleSlab)
    st.set_state(U)
    st.step(0.5, nsteps=2)
    Ur, _ = oracle.OracleGrid(spec).step(U, cfl=0.5, nsteps=2)
    got = st.get_state(np.zeros_like(U))
    assert np.max(np.abs(got - Ur).reshape(4, -1).max(axis=1) / np.abs(Ur).reshape(4, -1).max(axis=1)) < 1e-13


@pytest.mark.parametrize("overlap", [False, True])
def test_local_slabs_with_solid_ghost_rows(overlap):
    """Five slabs of the warped step (20 rows): the slab edges at rows 4 and 8 cut through the
    solid block's top (rows 0-3), so ghost rows hold solid cells and MUSCL stencils reach into
    them; the static ghost rows (mask, vertices) and the interior / edge split of every stage
    reproduce the whole grid."""
    import sys
    sys.path.insert(0, os.path.dirname(os.path.abspath(__file__)))
    import numpy as np
    import oracle
    from paper_1711_09272_gb300.slab import LocalExchange, SlabStepper, partition
    from slab_oracle import OracleSlab
    spec, U = _slab_case("warped_solid")
    slabs = partition(spec, 5)
    assert any(np.any(sl[4]["solid"].get(2, np.zeros(1))) for sl in slabs)
    st = SlabStepper(spec, 5, list(range(5)), LocalExchange(), make_slab=OracleSlab, overlap=overlap)
    st.set_state(U)
    dts = [st.step(0.5) for _ in range(2)]
    got = st.get_state(np.zeros_like(U))
    g = oracle.OracleGrid(spec)
    Ur = U.copy()
    for dt in dts:
        Ur, _ = g.step(Ur, dt_fixed=dt)
    scale = np.abs(Ur).reshape(4, -1).max(axis=1)[:, None, None]
    assert np.max(np.abs(got - Ur) / scale) < 1e-13
