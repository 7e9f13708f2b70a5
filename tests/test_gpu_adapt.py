"""Device criterion and adaptation vs the FP64 oracle, through the C ABI.

Integer results (trees, Morton keys, statuses through the trees they
produce) must be bit-exact.  The FP64 block norms agree within 1e-12 of the
field maximum (fused multiply-adds and separable sums on the device; the
same bound as the ghost fill), and the seeded fields keep every block norm
farther than that from both thresholds, so the decisions are unique and must
agree exactly.  FP64 adaptation fields are compared at 1e-12 relative; FP32
grids are compared against the oracle run on the same FP32 snapshot
(upcast), with FP64 ghosts on both sides.
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


def _tree():
    nt, tl = (4, 4, 4), 0.25
    lev, anc = I.uniform_leaves(nt, 0)
    lev, anc = I.refine_leaves(lev, anc, np.all((anc >= 1) & (anc <= 2), axis=1))
    lev, anc = I.refine_leaves(lev, anc, (lev == 1) & np.all(anc == 3, axis=1))
    lev, anc = I.balance(nt, lev, anc)
    return nt, tl, lev, anc


def _setup(mr, O, N, Nt, prec, lmax=3, cap=12000):
    nt, tl, lev, anc = _tree()
    nb = 16 if N < 6 else 24
    g = mr.Grid(nt, tl, nb, 0, lmax, N, Nt, lev, anc, precision=prec, capacity=cap)
    glev, ganc, _ = g.leaves()
    og = O.Grid(nt, tl, nb, N, Nt, 0, lmax, glev, ganc)
    xyz = I.point_coords(nt, tl, nb, glev, ganc)
    # a narrow blob in the coarse (level-0) region: leaves there refine, the
    # refined centre of the tree (levels 1-2) sees tiny details and coarsens
    phi = I.gaussian(xyz, (0.3, 0.3, 0.3), 0.05)
    if prec == mr.F32:
        phi = phi.astype(np.float32)
    g.field_copy_in(0, phi)
    return g, og, phi.astype(np.float64)


@pytest.mark.parametrize("N,Nt", [(2, 0), (4, 0), (4, 2), (6, 2)])
@pytest.mark.parametrize("prec", [0, 1])
def test_criterion_matches_oracle(mr, oracle_mod, N, Nt, prec):
    import torch
    O = oracle_mod
    g, og, phi = _setup(mr, O, N, Nt, prec)
    md = torch.empty(og.nleaf, dtype=torch.float64, device="cuda")
    g.criterion(0, md)
    g.sync()
    ref = O.block_maxdet(og, phi)
    assert np.abs(md.cpu().numpy() - ref).max() <= TOL * np.abs(phi).max()


TOL = 1e-12


def _eps(ref, phi=None):
    er, ec = 1e-3, 1e-7
    if phi is not None:
        _no_near_ties(ref, er, ec, phi)
    return er, ec


def _no_near_ties(maxdet, er, ec, phi):
    """Every block norm is farther than the FP64 tolerance from both
    thresholds, so the refine / coarsen decision of each block is unique."""
    tol = TOL * np.abs(phi).max()
    assert np.all(np.abs(maxdet - er) > tol) and np.all(np.abs(maxdet - ec) > tol)


@pytest.mark.parametrize("N,Nt", [(2, 0), (4, 0), (4, 2), (2, 2)])
def test_adapt_iteration_fp64_matches_oracle(mr, oracle_mod, N, Nt):
    O = oracle_mod
    g, og, phi = _setup(mr, O, N, Nt, mr.F64)
    er, ec = _eps(O.block_maxdet(og, phi), phi)
    nch = g.adapt_iter(0, er, ec)
    og2, ophi, _, onch, _, st = O.adapt_iter(og, phi, er, ec)
    assert nch == onch and nch > 0
    assert (st == 1).any()
    if Nt == 2 and N >= 4:  # narrow enough for the higher-order lifted wavelets to coarsen
        assert (st == -1).any()
    glev, ganc, gkeys = g.leaves()
    okeys = np.array([O.morton_key(l, *a, og.lmax) for l, a in zip(og2.lev, og2.anc)], np.uint64)
    assert np.array_equal(glev, og2.lev) and np.array_equal(ganc, og2.anc)
    assert np.array_equal(gkeys, okeys) and np.all(np.diff(gkeys.astype(np.float64)) > 0)
    got = g.field_copy_out(0)
    assert np.abs(got - ophi).max() <= TOL * np.abs(ophi).max()


@pytest.mark.parametrize("N,Nt", [(4, 2), (2, 0)])
def test_adapt_to_convergence_fp32_flags_exact(mr, oracle_mod, N, Nt):
    """Full Alg. SM3 loop on an FP32 grid: each iteration the oracle runs on
    the device's FP32 snapshot; statuses (through the trees) match exactly."""
    O = oracle_mod
    g, og, phi = _setup(mr, O, N, Nt, mr.F32)
    er, ec = _eps(O.block_maxdet(og, phi))
    refined = None
    for it in range(6):
        lev, anc, _ = g.leaves()
        cur = og.with_leaves(lev, anc)
        snap = g.field_copy_out(0).astype(np.float64)
        _no_near_ties(O.block_maxdet(cur, snap), er, ec, snap)
        og2, ophi, refined_o, onch, _, _ = O.adapt_iter(cur, snap, er, ec, refined)
        nch = g.adapt_iter(0, er, ec)
        assert nch == onch
        lev2, anc2, _ = g.leaves()
        assert np.array_equal(lev2, og2.lev) and np.array_equal(anc2, og2.anc)
        got = g.field_copy_out(0).astype(np.float64)
        assert np.abs(got - ophi).max() <= 2e-6 * max(1.0, np.abs(ophi).max())
        refined = refined_o
        if nch == 0:
            break
    assert it > 0


def test_mr_adapt_loop_fp64(mr, oracle_mod):
    O = oracle_mod
    g, og, phi = _setup(mr, O, 4, 2, mr.F64)
    er, ec = _eps(O.block_maxdet(og, phi))
    total = g.adapt(0, er, ec)
    og2, ophi, iters = O.adapt(og, phi, er, ec)
    lev, anc, _ = g.leaves()
    assert total > 0
    assert np.array_equal(lev, og2.lev) and np.array_equal(anc, og2.anc)
    got = g.field_copy_out(0)
    assert np.abs(got - ophi).max() <= TOL * np.abs(ophi).max()


def test_deformation_initial_grid_on_device(mr, oracle_mod):
    """Sec. 5.3 initial grid (compact Gaussian, 2.2, eps_r = 1e-2) built by the
    device's criterion, policy and refinement: the same 92 leaves on levels
    2 and 3 as the oracle and the paper."""
    nt, tl, nb, er = (1, 1, 1), 1.0, 24, 1e-2
    lev, anc = I.uniform_leaves(nt, 2)
    g = mr.Grid(nt, tl, nb, 2, 8, 2, 2, lev, anc, precision=mr.F64, capacity=1000)
    for _ in range(8):
        glev, ganc, _ = g.leaves()
        g.field_copy_in(0, I.compact_gaussian(I.point_coords(nt, tl, nb, glev, ganc)))
        if g.adapt_iter(0, er, er / 100, flags=mr.ADAPT_REFINE) == 0:
            break
    glev, ganc, _ = g.leaves()
    counts = np.bincount(glev, minlength=4)
    assert len(glev) == 92 and counts[2] == 60 and counts[3] == 32
    # the oracle's tree, leaf for leaf
    from test_oracle_pins import _deformation_initial_grid
    olev, oanc = _deformation_initial_grid(oracle_mod, 2, 2)
    key = lambda lv, an: sorted(zip(lv.tolist(), map(tuple, an.tolist())))
    assert key(glev, ganc) == key(olev, oanc)
