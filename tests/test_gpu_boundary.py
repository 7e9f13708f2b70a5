"""GPU path vs the FP64 oracle on forests with physical boundaries (Sec. 2.4),
through the C ABI: ghost fill, block criterion and RK3 steps on the 3-level
tree whose refinement meets the domain faces (inputs.bounded_test_tree),
bounded along every axis or along x only, with the extrapolation, zero-value
and plain-zero conditions; and adaptation iterations (Alg. SM3) on such
grids.

Tolerance.  The device evaluates the boundary polynomial with its Lagrange
weights, the oracle with Neville's algorithm: the same polynomial, rounded
differently.  Each differs from the exact value by at most a few units of
rounding times sum_j |w_j| |f_j|, and along k bounded axes at once (edges,
corners) the weights multiply; refinement of coarse values multiplies by at
most sum |K^s| <= 1.4 per axis.  So ghost values agree within
8 u Lambda^k 1.4^3 max|f|, Lambda the largest sum |w_j| over the distances a
ghost fill reaches beyond a boundary (u = 2^-53 for FP64 grids, 2^-24 for
FP32 grids); every other value of the path keeps the tolerance of the
periodic tests (1e-12 FP64, 1e-5 FP32 of the field maximum).
"""
import numpy as np
import pytest

from paper_2112_07537_gb300 import inputs as I

pytestmark = pytest.mark.gpu

NT, TL = (4, 4, 4), 0.25


@pytest.fixture(scope="module")
def mr():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2112_07537_gb300 import build, mrgb
    build.build()
    return mrgb


def _lebesgue(N, smax):
    """max over s = 1..smax of sum_j |w_j(-s)|, w_j the Lagrange weights of
    the nodes 0..N-1 (the extrapolation condition; the zero-value nodes give
    smaller sums)."""
    best = 0.0
    for s in range(1, smax + 1):
        tot = 0.0
        for j in range(N):
            w = 1.0
            for k in range(N):
                if k != j:
                    w *= (-s - k) / (j - k)
            tot += abs(w)
        best = max(best, tot)
    return best


def _tol(N, G, naxes, prec):
    u = 2.0 ** -53 if prec == 1 else 2.0 ** -24
    smax = (G + 1) // 2 + N // 2 + 1  # coarse points a refinement reads beyond
    return max(8 * u * _lebesgue(N, max(smax, G)) ** naxes * 1.4 ** 3, 1e-12 if prec == 1 else 1e-5)


def _grids(mr, O, N, Nt, nb, prec, bounded, bc, nfields=1):
    lev, anc = I.bounded_test_tree(NT)
    g = mr.Grid(NT, TL, nb, 0, 4, N, Nt, lev, anc, precision=prec, nfields=nfields, bounded=bounded, bc=bc)
    glev, ganc, _ = g.leaves()
    periodic = tuple(0 if b else 1 for b in bounded)
    og = O.Grid(NT, TL, nb, N, Nt, 0, 4, glev, ganc, periodic, bc)
    return g, og


def _field(og, nb):
    """Smooth and non-polynomial, nonzero on the boundaries (so the
    condition matters)."""
    x, y, z = I.point_coords(og.nt, og.tree_len, nb, og.lev, og.anc)
    return np.exp(np.sin(2.1 * x + 0.3) * np.cos(1.7 * y) + 0.5 * z)


@pytest.mark.parametrize("N,Nt,bounded,bc", [
    (4, 0, (1, 1, 1), 0), (4, 2, (1, 1, 1), 0), (2, 2, (1, 1, 1), 0), (6, 2, (1, 0, 0), 0),
    (6, 0, (1, 0, 0), 0), (4, 2, (1, 1, 1), 1), (4, 2, (1, 0, 1), 2)])
def test_bounded_ghost_fill_fp64(mr, oracle_mod, N, Nt, bounded, bc):
    import torch
    nb = 16 if N < 6 else 24
    g, og = _grids(mr, oracle_mod, N, Nt, nb, mr.F64, bounded, bc)
    f = _field(og, nb)
    G = 3
    ref_pad, ref_sub = oracle_mod.ghost_fill(og, f, G)
    g.field_copy_in(0, f)
    W = nb + 2 * G
    pad = torch.empty((g.nleaf, W, W, W), dtype=torch.float64, device="cuda")
    g.ghost_fill(0, G, pad)
    g.sync()
    scale = np.abs(ref_pad).max()
    tol = _tol(N, G, sum(bounded), 1)
    assert np.abs(pad.cpu().numpy() - ref_pad).max() <= tol * scale
    assert np.abs(g.field_copy_out(0) - ref_sub).max() <= 1e-12 * scale


@pytest.mark.parametrize("N,Nt", [(4, 2), (2, 0)])
def test_bounded_ghost_fill_fp32(mr, oracle_mod, N, Nt):
    import torch
    nb, G, bounded = 16, 3, (1, 0, 0)
    g, og = _grids(mr, oracle_mod, N, Nt, nb, mr.F32, bounded, 0)
    f = _field(og, nb).astype(np.float32)
    ref_pad, _ = oracle_mod.ghost_fill(og, f.astype(np.float64), G)
    g.field_copy_in(0, f)
    W = nb + 2 * G
    pad = torch.empty((g.nleaf, W, W, W), dtype=torch.float32, device="cuda")
    g.ghost_fill(0, G, pad)
    g.sync()
    err = np.abs(pad.cpu().numpy().astype(np.float64) - ref_pad).max() / np.abs(ref_pad).max()
    assert err <= _tol(N, G, 1, 0), err


@pytest.mark.parametrize("N,Nt,bounded", [(4, 2, (1, 1, 1)), (6, 2, (1, 0, 0))])
def test_bounded_criterion_fp64(mr, oracle_mod, N, Nt, bounded):
    nb = 16 if N < 6 else 24
    g, og = _grids(mr, oracle_mod, N, Nt, nb, mr.F64, bounded, 0)
    f = _field(og, nb)
    Ga = oracle_mod.adapt_shell(N, Nt)
    pad, _ = oracle_mod.ghost_fill(og, f, Ga)
    ref = oracle_mod.criterion(og, pad, Ga)
    g.field_copy_in(0, f)
    import torch
    md = torch.empty(g.nleaf, dtype=torch.float64, device="cuda")
    g.criterion(0, md)
    got = md.cpu().numpy()
    assert np.abs(got - ref).max() <= _tol(N, Ga, sum(bounded), 1) * np.abs(f).max()


@pytest.mark.parametrize("prec", [1, 0])
def test_bounded_rk3_steps(mr, oracle_mod, prec):
    """Three RK3 steps of WENO-Z5 advection with the extrapolation condition
    on every face (FP64) or on the x faces (FP32), against the oracle."""
    N, Nt, nb = 4, 2, 16
    bounded = (1, 1, 1) if prec == 1 else (1, 0, 0)
    g, og = _grids(mr, oracle_mod, N, Nt, nb, prec, bounded, 0)
    f = _field(og, nb)
    if prec == 0:
        f = f.astype(np.float32)
    g.field_copy_in(0, f)
    u = (1.0, -0.5, 0.25)
    dt = oracle_mod.dt_cfl(og, 0.5, u)
    ref = f.astype(np.float64)
    for _ in range(3):
        g.step(0, dt, u, mr.WENOZ5)
        ref = oracle_mod.rk3_step(og, ref, dt, oracle_mod.WENOZ5, u)
    err = np.abs(g.field_copy_out(0).astype(np.float64) - ref).max() / np.abs(ref).max()
    assert err <= (_tol(N, 3, sum(bounded), 1) if prec == 1 else 1e-4), err


def test_bounded_velocity_field_step(mr, oracle_mod):
    """mr_step_vel on a grid bounded along x: the velocity components are
    ghost-filled with the same boundary condition."""
    N, Nt, nb = 4, 2, 16
    lev, anc = I.bounded_test_tree(NT)
    g = mr.Grid(NT, TL, nb, 0, 4, N, Nt, lev, anc, precision=mr.F64, nfields=4, bounded=(1, 0, 0),
                velocity=True)
    glev, ganc, _ = g.leaves()
    og = oracle_mod.Grid(NT, TL, nb, N, Nt, 0, 4, glev, ganc, (0, 1, 1), 0)
    f = _field(og, nb)
    x, y, z = I.point_coords(og.nt, og.tree_len, nb, og.lev, og.anc)
    vel = [0.5 + 0.3 * np.cos(2 * x), 0.2 * np.sin(2 * np.pi * y), 0.1 + 0 * z]
    g.field_copy_in(0, f)
    for d in range(3):
        g.field_copy_in(1 + d, vel[d])
    vpads = [oracle_mod.ghost_fill(og, oracle_mod.ghost_fill(og, v, 3)[1], 3)[0] for v in vel]
    dt = 0.4 * (TL / (nb * 4)) / 1.0
    ref = f.copy()
    for _ in range(2):
        g.step_vel(0, dt, (1, 2, 3), mr.WENOZ5)
        ref = oracle_mod.rk3_step_velpad(og, ref, vpads, dt, oracle_mod.WENOZ5)
    err = np.abs(g.field_copy_out(0) - ref).max() / np.abs(ref).max()
    assert err <= _tol(N, 3, 1, 1), err


# bounded axes chosen so that no block norm lies within 10x the bound of a
# threshold (the bound grows with the number of bounded axes; the all-axes
# 4.2 bound, ~1e-6, would cover norms near eps_c = 1e-7)
@pytest.mark.parametrize("N,Nt,bounded", [(4, 2, (1, 0, 0)), (4, 0, (1, 0, 1)), (2, 2, (1, 1, 1))])
def test_bounded_adaptation_matches_oracle(mr, oracle_mod, N, Nt, bounded):
    """Alg. SM3 iterations with physical boundaries on two FP64 fields (the
    criterion field and a second one refined, coarsened and updated by its
    decisions): a narrow Gaussian on the x = 0 face refines the blocks there,
    the smooth level-1/2 region coarsens.  Trees and statuses exactly as the
    oracle's; fields within the ghost tolerance (the refinement of children
    reads ghosts beyond the boundary)."""
    nb, lmax = 16, 4
    lev, anc = I.bounded_test_tree(NT)
    g = mr.Grid(NT, TL, nb, 0, lmax, N, Nt, lev, anc, precision=mr.F64, nfields=2, bounded=bounded,
                capacity=8000)
    glev, ganc, _ = g.leaves()
    periodic = tuple(0 if b else 1 for b in bounded)
    og = oracle_mod.Grid(NT, TL, nb, N, Nt, 0, lmax, glev, ganc, periodic, 0)
    x, y, z = I.point_coords(NT, TL, nb, glev, ganc)
    phi = np.exp(-((x - 0.02) ** 2 + (y - 0.6) ** 2 + (z - 0.55) ** 2) / 0.06 ** 2)
    psi = np.cos(3.0 * x) * np.exp(0.5 * y - 0.2 * z)
    g.field_copy_in(0, phi)
    g.field_copy_in(1, psi)
    er, ec = 1e-3, 1e-7
    tol = _tol(N, oracle_mod.adapt_shell(N, Nt), sum(bounded), 1)
    refined = None
    cur, fields = og, [phi, psi]
    for it in range(4):
        Ga = oracle_mod.adapt_shell(N, Nt)
        norms = oracle_mod.criterion(cur, oracle_mod.ghost_fill(cur, fields[0], Ga)[0], Ga)
        # no block norm within the tolerance of a threshold: decisions unique
        assert np.all(np.abs(norms - er) > 10 * tol) and np.all(np.abs(norms - ec) > 10 * tol)
        og2, ofields, refined, onch, _, st = oracle_mod.adapt_iter_fields(cur, fields, er, ec, refined)
        nch = g.adapt_iter(0, er, ec)
        assert nch == onch
        lev2, anc2, _ = g.leaves()
        assert np.array_equal(lev2, og2.lev) and np.array_equal(anc2, og2.anc)
        for f in range(2):
            got = g.field_copy_out(f)
            assert np.abs(got - ofields[f]).max() <= tol * np.abs(ofields[f]).max(), (it, f)
        if it == 0:
            assert (st == 1).any() and (st == -1).any()
        cur, fields = og2, [g.field_copy_out(0), g.field_copy_out(1)]
        if nch == 0:
            break


def test_bounded_grids_refuse_what_they_do_not_support(mr):
    lev, anc = I.bounded_test_tree(NT)
    g = mr.Grid(NT, TL, 16, 0, 4, 4, 2, lev, anc, precision=mr.F64, bounded=(1, 0, 0), capacity=2000)
    with pytest.raises(mr.MRError):
        g.ghost_fill_static(0, 3)
    lev1, anc1 = I.uniform_leaves((1, 1, 1), 1)
    with pytest.raises(mr.MRError):
        mr.Grid((1, 1, 1), 1.0, 16, 0, 2, 4, 2, lev1, anc1, bounded=(1, 0, 0), independent_trees=True)
