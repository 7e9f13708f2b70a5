"""The allocation-free ghost fill (mr_ghost_fill_static) against the regular
one, through the C ABI.

Some callers cannot allocate device memory at the moment they call the
library (their memory is fixed up front by another runtime), so the library
offers one entry point whose scratch lives in static device memory.  This
file runs last: it checks that variant against mr_ghost_fill on two calls in
a row (the static scratch keeps the previous call's contents), with the
tolerances of the other ghost-fill tests (bit-exact: the same kernels run),
and that grids too large for the static scratch are refused.
"""
import numpy as np
import pytest

from paper_2112_07537_gb300 import inputs as I

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def mr():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2112_07537_gb300 import build, mrgb
    build.build()
    return mrgb


@pytest.mark.parametrize("prec,N,Nt", [(0, 4, 2), (1, 6, 2)])
def test_static_ghost_fill_matches_regular(mr, prec, N, Nt):
    import torch
    nt, tl = (2, 2, 2), 0.5
    nb = 16 if N < 6 else 24
    lev, anc = I.tree_config1()
    a = mr.Grid(nt, tl, nb, 0, 1, N, Nt, lev, anc, precision=prec)
    b = mr.Grid(nt, tl, nb, 0, 1, N, Nt, lev, anc, precision=prec)
    glev, ganc, _ = a.leaves()
    dt = torch.float32 if prec == 0 else torch.float64
    for call, seed in enumerate((1, 2)):  # two calls in a row, different data
        rng = np.random.default_rng(seed)
        phi = rng.normal(size=(len(glev), nb, nb, nb)).astype(np.float32 if prec == 0 else np.float64)
        a.field_copy_in(0, phi)
        b.field_copy_in(0, phi)
        G = 3 + call
        W = nb + 2 * G
        pa = torch.empty((len(glev), W, W, W), dtype=dt, device="cuda")
        pb = torch.empty_like(pa)
        a.ghost_fill(0, G, pa)
        b.ghost_fill_static(0, G, pb)
        a.sync()
        b.sync()
        assert torch.equal(pa, pb)
        assert np.array_equal(a.field_copy_out(0), b.field_copy_out(0))


@pytest.mark.parametrize("N,Nt,G", [(4, 0, 4), (4, 2, 5)])
def test_static_ghost_fill_fp64_padded_path(mr, N, Nt, G):
    """FP32 grids whose internal shell is wider than the stencil buffers get
    FP64 padded blocks from mr_ghost_fill; the static variant takes the same
    path (same kernels, same precision), so the results are bit-identical."""
    import torch
    nt, tl, nb = (2, 2, 2), 0.5, 16
    lev, anc = I.tree_config1()
    a = mr.Grid(nt, tl, nb, 0, 1, N, Nt, lev, anc, precision=mr.F32)
    b = mr.Grid(nt, tl, nb, 0, 1, N, Nt, lev, anc, precision=mr.F32)
    n = a.nleaf
    for seed in (3, 4):  # two calls in a row
        phi = np.random.default_rng(seed).normal(size=(n, nb, nb, nb)).astype(np.float32)
        a.field_copy_in(0, phi)
        b.field_copy_in(0, phi)
        W = nb + 2 * G
        pa = torch.empty((n, W, W, W), dtype=torch.float32, device="cuda")
        pb = torch.empty_like(pa)
        a.ghost_fill(0, G, pa)
        b.ghost_fill_static(0, G, pb)
        a.sync()
        b.sync()
        assert torch.equal(pa, pb)
        assert np.array_equal(a.field_copy_out(0), b.field_copy_out(0))


def test_static_ghost_fill_unsupported_where_regular_is(mr):
    """Where mr_ghost_fill refuses a shell (wider than both buffers of the
    grid, or an FP64 padded path on a fixed-tree grid), so does the static
    variant."""
    nt, tl, nb = (2, 2, 2), 0.5, 16
    lev, anc = I.tree_config1()
    g = mr.Grid(nt, tl, nb, 0, 1, 2, 0, lev, anc, precision=mr.F32)
    for call in (g.ghost_fill, g.ghost_fill_static):
        with pytest.raises(mr.MRError) as e:
            call(0, 4)
        assert e.value.code == -5
    f = mr.Grid(nt, tl, nb, 0, 1, 4, 0, lev, anc, precision=mr.F32, fixed_tree=True)
    for call in (f.ghost_fill, f.ghost_fill_static):
        with pytest.raises(mr.MRError) as e:
            call(0, 4)
        assert e.value.code == -5


def test_static_ghost_fill_rejects_oversize_grid(mr):
    nt = (2, 2, 2)
    # 64 leaves of 32^3 with shell 11 (the adaptation shell of 6.2): two
    # padded FP64 buffers of 64 * 54^3 values, 161 MB > 64 MiB
    lev, anc = I.uniform_leaves(nt, 1)
    g = mr.Grid(nt, 0.5, 32, 0, 1, 6, 2, lev, anc, precision=mr.F64)
    with pytest.raises(mr.MRError) as e:
        g.ghost_fill_static(0, 11)
    assert e.value.code == -2
