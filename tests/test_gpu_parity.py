"""GPU path vs the FP64 oracle, element by element, through the C ABI.

Tolerances: FP64 ghost fill within 1e-12 of the field maximum (the device
sums with fused multiply-adds and evaluates the Part-2 coarsening
separably; a sum of n <= 729 terms with weights of absolute sum <= 14 in 3D
errs by at most n * 2^-53 * 14 * max|phi| ~ 1e-12 * max|phi|, typically
1e-15); FP64 stencils and RK3 steps within 1e-12 relative to the field
maximum; FP32 within 1e-5 of the field maximum (rounding of ~1e2 FP32
operations per point per stage).
"""
import numpy as np
import pytest

from paper_2112_07537_gb300 import inputs as I

pytestmark = pytest.mark.gpu

WAV = [(2, 0), (2, 2), (4, 0), (4, 2), (6, 0), (6, 2)]
FP64_GHOST_TOL = 1e-12


@pytest.fixture(scope="module")
def mr():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2112_07537_gb300 import build, mrgb
    build.build()
    mrgb.load()
    return mrgb


def _sorted_by_oracle_keys(O, lev, anc, kl):
    keys = np.array([O.morton_key(l, *a, kl) for l, a in zip(lev, anc)], dtype=np.uint64)
    order = np.argsort(keys, kind="stable")
    return lev[order], anc[order], keys[order]


def _three_level(nb):
    nt, tl = (4, 4, 4), 0.25
    lev, anc = I.uniform_leaves(nt, 0)
    lev, anc = I.refine_leaves(lev, anc, np.all((anc >= 1) & (anc <= 2), axis=1))
    lev, anc = I.refine_leaves(lev, anc, (lev == 1) & np.all(anc == 3, axis=1))
    lev, anc = I.balance(nt, lev, anc)
    return nt, tl, lev, anc


def _grid(mr, O, nt, tl, nb, N, Nt, lev, anc, prec, lmax, nfields=1, cap=None):
    g = mr.Grid(nt, tl, nb, 0, lmax, N, Nt, lev, anc, precision=prec, nfields=nfields, capacity=cap)
    glev, ganc, gkeys = g.leaves()
    olev, oanc, okeys = _sorted_by_oracle_keys(O, lev, anc, lmax)
    # S0: the device's Morton order and keys equal the oracle's, bit for bit
    assert np.array_equal(glev, olev) and np.array_equal(ganc, oanc)
    assert np.array_equal(gkeys, okeys)
    og = O.Grid(nt, tl, nb, N, Nt, 0, lmax, glev, ganc)
    return g, og


@pytest.mark.parametrize("N,Nt", WAV)
def test_ghost_fill_fp64(mr, oracle_mod, N, Nt):
    O = oracle_mod
    nb = 16 if N < 6 else 24
    nt, tl, lev, anc = _three_level(nb)
    g, og = _grid(mr, O, nt, tl, nb, N, Nt, lev, anc, mr.F64, 2)
    rng = np.random.default_rng(100 + N + Nt)
    phi = rng.normal(size=(og.nleaf, nb, nb, nb))
    import torch
    for G in sorted({3, O.adapt_shell(N, Nt)}):
        g.field_copy_in(0, phi)
        W = nb + 2 * G
        pad = torch.empty((og.nleaf, W, W, W), dtype=torch.float64, device="cuda")
        g.ghost_fill(0, G, pad)
        g.sync()
        ref_pad, ref_sub = O.ghost_fill(og, phi, G)
        tol = FP64_GHOST_TOL * np.abs(phi).max()
        err = np.abs(pad.cpu().numpy() - ref_pad).max()
        assert err <= tol, (G, err)
        assert np.abs(g.field_copy_out(0) - ref_sub).max() <= tol


@pytest.mark.parametrize("N,Nt", [(4, 0), (4, 2), (6, 2)])
def test_ghost_fill64_of_fp32_field(mr, oracle_mod, N, Nt):
    """The adaptation path: FP64 ghosts from an FP32 field equal the oracle's
    ghosts of the same (upcast) values."""
    O = oracle_mod
    nb = 16 if N < 6 else 24
    nt, tl, lev, anc = _three_level(nb)
    g, og = _grid(mr, O, nt, tl, nb, N, Nt, lev, anc, mr.F32, 2)
    rng = np.random.default_rng(7)
    phi = rng.normal(size=(og.nleaf, nb, nb, nb)).astype(np.float32)
    g.field_copy_in(0, phi)
    G = O.adapt_shell(N, Nt)
    import torch
    W = nb + 2 * G
    pad = torch.empty((og.nleaf, W, W, W), dtype=torch.float64, device="cuda")
    g.ghost_fill64(0, G, pad)
    g.sync()
    ref_pad, ref_sub = O.ghost_fill(og, phi.astype(np.float64), G)
    tol = FP64_GHOST_TOL * np.abs(phi).max()
    assert np.abs(pad.cpu().numpy() - ref_pad).max() <= tol
    # the substituted interior is stored back in FP32: one rounding
    got = g.field_copy_out(0).astype(np.float64)
    assert np.abs(got - ref_sub).max() <= 2.0 ** -24 * np.abs(ref_sub).max() + tol


@pytest.mark.parametrize("N,Nt", [(2, 0), (4, 2), (6, 2)])
def test_ghost_fill_fp32_tolerance(mr, oracle_mod, N, Nt):
    O = oracle_mod
    nb = 16 if N < 6 else 24
    nt, tl, lev, anc = _three_level(nb)
    g, og = _grid(mr, O, nt, tl, nb, N, Nt, lev, anc, mr.F32, 2)
    xyz = I.point_coords(nt, tl, nb, og.lev, og.anc)
    phi = I.fourier_front(xyz, seed=3, kmax=4, width=0.05).astype(np.float32)
    g.field_copy_in(0, phi)
    import torch
    W = nb + 6
    pad = torch.empty((og.nleaf, W, W, W), dtype=torch.float32, device="cuda")
    g.ghost_fill(0, 3, pad)
    g.sync()
    ref_pad, _ = O.ghost_fill(og, phi.astype(np.float64), 3)
    # FP32 sums of up to 26 terms with sum|w| <= 14: a few 1e-6 of the field max
    scale = np.abs(ref_pad).max()
    assert np.abs(pad.cpu().numpy() - ref_pad).max() <= 1e-5 * scale


@pytest.mark.parametrize("scheme", [0, 1, 2])
@pytest.mark.parametrize("prec", [0, 1])
def test_rhs_parity(mr, oracle_mod, scheme, prec):
    O = oracle_mod
    nt, tl, nb = (2, 2, 2), 0.5, 16
    lev, anc = I.tree_config1()
    g, og = _grid(mr, O, nt, tl, nb, 4, 0, lev, anc, prec, 1, nfields=2)
    xyz = I.point_coords(nt, tl, nb, og.lev, og.anc)
    phi = I.gaussian_images(xyz, (0.45, 0.55, 0.5), 0.1, nimg=1)
    if prec == 0:
        phi = phi.astype(np.float32)
    g.field_copy_in(0, phi)
    u = (1.0, -0.5, 0.25)
    g.rhs_advect(0, u, 1, scheme)
    got = g.field_copy_out(1).astype(np.float64)
    pad, _ = O.ghost_fill(og, phi.astype(np.float64), 3)
    ref = O.rhs(og, pad, 3, scheme, u)
    tol = 1e-12 if prec == 1 else 2e-5
    assert np.abs(got - ref).max() <= tol * np.abs(ref).max()


def test_rk_stage_elementwise(mr, oracle_mod):
    nt, tl, nb = (2, 2, 2), 0.5, 16
    lev, anc = I.tree_config1()
    g = mr.Grid(nt, tl, nb, 0, 1, 4, 0, lev, anc, precision=mr.F64, nfields=4)
    rng = np.random.default_rng(5)
    a, b, c = (rng.normal(size=(g.nleaf, nb, nb, nb)) for _ in range(3))
    for fid, x in enumerate((a, b, c)):
        g.field_copy_in(fid, x)
    for stage, ref in ((0, b + 0.1 * c), (1, 0.75 * a + 0.25 * (b + 0.1 * c)),
                       (2, a / 3 + 2.0 / 3 * (b + 0.1 * c))):
        g.rk_stage(stage, 0.1, 0, 1, 2, 3)
        assert np.allclose(g.field_copy_out(3), ref, rtol=1e-14, atol=1e-14)


@pytest.mark.parametrize("prec,scheme", [(1, 2), (1, 1), (0, 2), (0, 1)])
def test_config1_ten_steps(mr, oracle_mod, prec, scheme):
    """Tiny configuration: 2x2x2 trees, one refined (15 leaves of 16^3), 4.0
    wavelet, Gaussian sigma=0.1 at the centre, u=(1,1,1), RK3, CFL 0.5,
    10 steps, fixed tree: GPU vs oracle after every step."""
    O = oracle_mod
    nt, tl, nb = (2, 2, 2), 0.5, 16
    lev, anc = I.tree_config1()
    g, og = _grid(mr, O, nt, tl, nb, 4, 0, lev, anc, prec, 1)
    xyz = I.point_coords(nt, tl, nb, og.lev, og.anc)
    phi = I.gaussian(xyz, (0.5, 0.5, 0.5), 0.1)
    if prec == 0:
        phi = phi.astype(np.float32)
    g.field_copy_in(0, phi)
    u = (1.0, 1.0, 1.0)
    dt = O.dt_cfl(og, 0.5, u)
    ref = phi.astype(np.float64)
    m0 = O.moments(og, ref)[0]
    for _ in range(10):
        g.step(0, dt, u, scheme)
        ref = O.rk3_step(og, ref, dt, scheme, u)
    got = g.field_copy_out(0).astype(np.float64)
    err = np.abs(got - ref).max() / np.abs(ref).max()
    assert err <= (1e-12 if prec == 1 else 1e-5), err
    # FP64 mass on the device matches the oracle quadrature of the same field
    assert g.mass(0) == pytest.approx(O.moments(og, got)[0], rel=1e-12)
    del m0


def test_invalid_trees_are_rejected(mr):
    nt = (1, 1, 1)
    lev, anc = I.uniform_leaves(nt, 1)
    # refine one leaf twice -> 2-level jump next to level-1 leaves
    lev, anc = I.refine_leaves(lev, anc, np.arange(len(lev)) == 0)
    lev, anc = I.refine_leaves(lev, anc, np.arange(len(lev)) == 0)
    with pytest.raises(mr.MRError) as e:
        mr.Grid(nt, 1.0, 16, 0, 3, 4, 0, lev, anc)
    assert e.value.code == -6
    lev2, anc2 = I.uniform_leaves(nt, 1)
    with pytest.raises(mr.MRError):  # a missing leaf leaves a hole
        mr.Grid(nt, 1.0, 16, 0, 3, 4, 0, lev2[1:], anc2[1:])


def _tg(xyz, comp, s=1.0, ph=0.3):
    """Taylor-Green-like divergence-free velocity component (comp 0, 1, 2)."""
    w = 2 * np.pi
    x, y, z = xyz
    if comp == 0:
        return s * np.sin(w * x + ph) * np.cos(w * y) * np.cos(w * z)
    if comp == 1:
        return -s * np.cos(w * x + ph) * np.sin(w * y) * np.cos(w * z)
    return np.zeros_like(x)


@pytest.mark.parametrize("prec", [1, 0])
@pytest.mark.parametrize("scheme", [1, 2])
def test_velocity_field_rhs_and_steps(mr, oracle_mod, prec, scheme):
    """Advection by grid velocity fields (u, v, w ghost-filled like phi,
    interface velocity (u_i + u_{i+1})/2 picks the upwind side): rhs and
    three RK3 steps against the oracle.  The device ghost-fills the (time
    independent) velocity once per tree -- substitute, then fill -- and the
    oracle steps with the same fixed velocity ghosts; refilling every stage
    as well would move values by ~1e-10 through repeated substitution of
    neighbouring bands."""
    O = oracle_mod
    nt, tl, nb = (2, 2, 2), 0.5, 16
    lev, anc = I.tree_config1()
    g = mr.Grid(nt, tl, nb, 0, 1, 6, 2, lev, anc, precision=prec, nfields=5, velocity=True)
    glev, ganc, _ = g.leaves()
    og = O.Grid(nt, tl, nb, 6, 2, 0, 1, glev, ganc)
    xyz = I.point_coords(nt, tl, nb, glev, ganc)
    phi = I.gaussian_images(xyz, (0.45, 0.5, 0.55), 0.1, nimg=1)
    vel = [_tg(xyz, d) for d in range(3)]
    cast = (lambda a: a.astype(np.float32)) if prec == 0 else (lambda a: a)
    g.field_copy_in(0, cast(phi))
    for d in range(3):
        g.field_copy_in(1 + d, cast(vel[d]))
    phi64 = cast(phi).astype(np.float64)
    # the device substitutes the velocity once per tree (idempotent); start
    # the oracle from the substituted velocity too
    vel64 = [O.ghost_fill(og, cast(v).astype(np.float64), 3)[1] for v in vel]
    vpads = [O.ghost_fill(og, v, 3)[0] for v in vel64]
    # rhs
    g.rhs_advect_vel(0, (1, 2, 3), 4, scheme)
    got = g.field_copy_out(4).astype(np.float64)
    pad, _ = O.ghost_fill(og, phi64, 3)
    ref = O.rhs(og, pad, 3, scheme, vel=vpads)
    tol = 1e-12 if prec == 1 else 2e-5
    assert np.abs(got - ref).max() <= tol * np.abs(ref).max()
    # steps (fresh copies: the rhs call substituted phi in place on both sides)
    g.field_copy_in(0, cast(phi))
    ref = phi64
    dt = 0.5 * (0.5 / (nb * 2)) / 2.0
    for _ in range(3):
        g.step_vel(0, dt, (1, 2, 3), scheme)
        ref = O.rk3_step_velpad(og, ref, vpads, dt, scheme)
    err = np.abs(g.field_copy_out(0).astype(np.float64) - ref).max() / np.abs(ref).max()
    assert err <= (1e-12 if prec == 1 else 1e-5), err


def test_profile_bytes_of_a_full_ghost_fill(mr, oracle_mod):
    """The ghost pre-pass's algorithmic bytes (roofline numerator): every
    point of the requested shell of every leaf's padded block written once
    and its source value read once."""
    import torch
    O = oracle_mod
    nb, N, Nt, G = 16, 4, 2, 3
    nt, tl, lev, anc = _three_level(nb)
    g, og = _grid(mr, O, nt, tl, nb, N, Nt, lev, anc, mr.F32, 2)
    g.field_copy_in(0, np.zeros((og.nleaf, nb, nb, nb), np.float32))
    W = nb + 2 * G
    pad = torch.empty((og.nleaf, W, W, W), dtype=torch.float32, device="cuda")
    g.profile(True)
    g.ghost_fill(0, G, pad)
    g.sync()
    # leaves with a coarser neighbour go through the full pre-pass (id 0),
    # the others through the plain gather (id 1): every leaf exactly once
    prep, plain = g.profile_bytes(0), g.profile_bytes(1)
    g.profile(False)
    Wd = nb + 2 * G  # the requested shell (the internal one counts as time)
    unit = (Wd ** 3 - nb ** 3) * (4 + 4)
    assert prep + plain == og.nleaf * unit
    assert prep > 0 and plain > 0 and prep % unit == 0
    assert g.profile_bytes(5) == 0.0


@pytest.mark.parametrize("order", [2, 4])
@pytest.mark.parametrize("prec", [1, 0])
def test_advection_diffusion_rhs_and_steps(mr, oracle_mod, prec, order):
    """DIFF-2 / DIFF-4 (Sec. 4.3) added to the WENO-Z5 advection right-hand
    side: rhs and three RK3 steps against the oracle on the two-level tree.
    FP32 tolerance: the Laplacian scales a ghost or rounding error of
    ~1e-6 max|phi| by at most 64/12 / h^2, and its own size here is
    >= 0.1 max|phi| / h^2, so a few 1e-5 of the right-hand side's maximum."""
    O = oracle_mod
    nt, tl, nb = (2, 2, 2), 0.5, 16
    lev, anc = I.tree_config1()
    g, og = _grid(mr, O, nt, tl, nb, 4, 2, lev, anc, prec, 1, nfields=2)
    xyz = I.point_coords(nt, tl, nb, og.lev, og.anc)
    phi = I.gaussian_images(xyz, (0.45, 0.55, 0.5), 0.1, nimg=1)
    if prec == 0:
        phi = phi.astype(np.float32)
    nu, u = 0.01, (1.0, -0.5, 0.25)
    g.set_diffusion(nu, order)
    g.field_copy_in(0, phi)
    g.rhs_advect(0, u, 1, mr.WENOZ5)
    got = g.field_copy_out(1).astype(np.float64)
    pad, _ = O.ghost_fill(og, phi.astype(np.float64), 3)
    ref = O.rhs(og, pad, 3, O.WENOZ5, u) + nu * O.laplacian(og, pad, 3, order)
    tol = 1e-12 if prec == 1 else 5e-5
    assert np.abs(got - ref).max() <= tol * np.abs(ref).max()
    # three steps (fresh copy: the rhs call substituted phi in place)
    g.field_copy_in(0, phi)
    h = tl / (nb * 2)
    dt = min(O.dt_cfl(og, 0.5, u), 0.1 * h * h / nu)
    ref = phi.astype(np.float64)
    for _ in range(3):
        g.step(0, dt, u, mr.WENOZ5)
        ref = O.rk3_step_diff(og, ref, dt, O.WENOZ5, u, nu, order)
    err = np.abs(g.field_copy_out(0).astype(np.float64) - ref).max() / np.abs(ref).max()
    assert err <= (1e-12 if prec == 1 else 1e-5), err
    # the term is removed again
    g.set_diffusion(0.0, 0)
    g.field_copy_in(0, phi)
    g.rhs_advect(0, u, 1, mr.WENOZ5)
    pad, _ = O.ghost_fill(og, phi.astype(np.float64), 3)
    ref = O.rhs(og, pad, 3, O.WENOZ5, u)
    assert np.abs(g.field_copy_out(1).astype(np.float64) - ref).max() <= tol * np.abs(ref).max()


@pytest.mark.parametrize("prec", [1, 0])
def test_time_dependent_velocity_steps(mr, oracle_mod, prec):
    """Sec. 5.3 workload pieces: the device-evaluated deformation field and
    compact Gaussian equal the host formulas, and RK3 steps with the stage
    scales of a time-dependent velocity (one of them negative) match the
    oracle."""
    O = oracle_mod
    nt, tl, nb = (2, 2, 2), 0.5, 16
    lev, anc = I.tree_config1()
    g = mr.Grid(nt, tl, nb, 0, 1, 4, 2, lev, anc, precision=prec, nfields=4, velocity=True)
    glev, ganc, _ = g.leaves()
    og = O.Grid(nt, tl, nb, 4, 2, 0, 1, glev, ganc)
    xyz = I.point_coords(nt, tl, nb, glev, ganc)
    g.field_set(0, mr.INIT_COMPACT_GAUSSIAN, [0.35, 0.35, 0.35, 0.1, 0.2, 1.0])
    for d in range(3):
        g.field_set(1 + d, mr.INIT_DEFORMATION, [d, 1.0])
    itol = 1e-13 if prec == 1 else 1e-6
    phi = I.compact_gaussian(xyz)
    assert np.abs(g.field_copy_out(0).astype(np.float64) - phi).max() <= itol
    vel = [I.deformation_velocity(xyz, d) for d in range(3)]
    for d in range(3):
        assert np.abs(g.field_copy_out(1 + d).astype(np.float64) - vel[d]).max() <= 2 * itol
    # the oracle starts from the device's own values (FP32 rounding included)
    phi64 = g.field_copy_out(0).astype(np.float64)
    v64 = [O.ghost_fill(og, g.field_copy_out(1 + d).astype(np.float64), 3)[1] for d in range(3)]
    vpads = [O.ghost_fill(og, v, 3)[0] for v in v64]
    h = tl / (nb * 2)
    dt = 0.25 * h / 3.0
    ref = phi64
    # stage scales with sign changes within and between steps (the factor
    # cos(pi t / 3) of Sec. 5.3 changes sign at t = 1.5)
    for sc in ((0.8, -0.6, 0.3), (-1.0, -0.2, 0.5), (1.2, 0.9, -0.7)):
        g.step_vel_scaled(0, dt, (1, 2, 3), mr.WENOZ5, sc)
        ref = O.rk3_step_velpad_scaled(og, ref, vpads, dt, O.WENOZ5, sc)
    err = np.abs(g.field_copy_out(0).astype(np.float64) - ref).max() / np.abs(ref).max()
    assert err <= (1e-12 if prec == 1 else 1e-5), err
