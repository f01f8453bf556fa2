"""The C-ABI library builds, loads and exports every entry point include/roeam.h and
include/roeam3.h declare (no compute calls: this runs without a GPU)."""
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    names = set()
    for h in ("roeam.h", "roeam3.h"):
        text = open(os.path.join(ROOT, "include", h)).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        names |= set(re.findall(r"\b(roeam3?_[a-z0-9_]+)\s*\(", text))
    return sorted(names)


def test_library_builds_and_exports_header_symbols():
    from paper_1711_09272_gb300 import build as b
    path = b.build()
    assert os.path.exists(path)
    import ctypes
    lib = ctypes.CDLL(path)
    names = declared_functions()
    assert "roeam_create_grid" in names and "roeam_rk_step" in names
    for n in names:
        assert hasattr(lib, n), n


def test_binding_names_match_header():
    import paper_1711_09272_gb300 as P
    assert sorted(P.EXPORTS) == declared_functions()
    lib = P.load_library()
    assert P.roeam_version() >= 10000
    assert lib.roeam_last_error() is not None


def test_create_rejects_bad_arguments_without_gpu_work():
    """Argument validation happens before any device call."""
    import workloads as W
    import paper_1711_09272_gb300 as P
    spec = W.GridSpec(ni=3, nj=8)
    with pytest.raises(P.RoeamError) as e:
        P.roeam_create_grid([P.make_desc(spec)])
    assert e.value.status == 1 and "ni, nj" in str(e.value)
    spec = W.GridSpec(ni=8, nj=8, bc=(W.PERIODIC, W.WALL, W.PERIODIC, W.PERIODIC))
    with pytest.raises(P.RoeamError) as e:
        P.roeam_create_grid([P.make_desc(spec)])
    assert "PERIODIC" in str(e.value)
    spec = W.with_params(W.GridSpec(ni=8, nj=8), gamma=1.0)
    with pytest.raises(P.RoeamError):
        P.roeam_create_grid([P.make_desc(spec)])
    a = P.make_desc(W.GridSpec(ni=8, nj=8), precision=32)
    b = P.make_desc(W.GridSpec(ni=8, nj=8), precision=64)
    with pytest.raises(P.RoeamError) as e:
        P.roeam_create_grid([a, b])
    assert "precision" in str(e.value)
    for kw, word in ((dict(scheme=2), "scheme"), (dict(dup_mode=3), "dup_mode"), (dict(harten=0.1), "harten"),
                     (dict(scheme=1, dup_mode=1), "Roe-AM variants"), (dict(scheme=1, harten=1.0), "harten"),
                     (dict(xi_roe=2), "xi_roe")):
        with pytest.raises(P.RoeamError) as e:
            P.roeam_create_grid([P.make_desc(W.with_params(W.GridSpec(ni=8, nj=8), **kw))])
        assert e.value.status == 1 and word in str(e.value), (kw, str(e.value))


def test_exchange_sides_are_validated():
    """EXCHANGE (row slabs) is accepted on S/N only, with or without solid cells."""
    import numpy as np
    import workloads as W
    import paper_1711_09272_gb300 as P
    for bc in ((4, W.OUTFLOW, W.WALL, W.WALL), (W.OUTFLOW, 4, W.WALL, W.WALL)):
        for solid in (None, np.zeros((8, 8), np.uint8)):
            spec = W.GridSpec(ni=8, nj=8, bc=bc)
            spec.solid = solid
            with pytest.raises(P.RoeamError) as e:
                P.roeam_create_grid([P.make_desc(spec)])
            assert "EXCHANGE" in str(e.value)


def test_size_limits_are_validated():
    """The largest handle holds 65535 grids of at most 2^28 cells each (the kernels index a
    grid's planes with 32-bit offsets); one grid more, or one cell row more, is refused before
    any device work, and so is an empty batch."""
    import workloads as W
    import paper_1711_09272_gb300 as P
    with pytest.raises(P.RoeamError) as e:
        P.roeam_create_grid([])
    assert e.value.status == 1 and "count" in str(e.value)
    with pytest.raises(P.RoeamError) as e:
        P.roeam_create_grid([P.make_desc(W.GridSpec(ni=4, nj=4))] * 65536)
    assert e.value.status == 1 and "65535" in str(e.value)
    with pytest.raises(P.RoeamError) as e:
        P.roeam_create_grid([P.make_desc(W.GridSpec(ni=16384, nj=16385))])
    assert e.value.status == 1 and "too many cells" in str(e.value)
    # the 3D handle has the same limits
    with pytest.raises(P.RoeamError) as e:
        P.roeam3_create_grid([P.make_desc3(W.GridSpec3(ni=4, nj=4, nk=4))] * 65536)
    assert e.value.status == 1 and "65535" in str(e.value)
    with pytest.raises(P.RoeamError) as e:
        P.roeam3_create_grid([P.make_desc3(W.GridSpec3(ni=1024, nj=1024, nk=257))])
    assert e.value.status == 1 and "too many cells" in str(e.value)
