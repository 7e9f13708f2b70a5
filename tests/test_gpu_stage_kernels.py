"""The two FP32 stage kernels against each other and against the FP64 oracle,
through the C ABI (mr_set_stage_kernel): k_fused holds the ghost-extended
block of a leaf in shared memory and walks grid lines, k_march traverses the
block plane by plane with a register window along z.  Both evaluate the same
interface fluxes (Tables SM3 / SM4, upwind by the interface velocity), the
same Laplacian (Sec. 4.3) and the same RK3-TVD stage combination on the same
ghost values, operation for operation, so their results may differ only where
the compiler contracts a product into a fused multiply-add differently: they
are compared at 1e-6 of the field maximum (in practice identical), and each
against the oracle at the FP32 tolerance of the other tests, 1e-5 of the
field maximum.  The trees have same-level, coarser and finer faces on every
leaf kind (the refined tree of the tiny configuration, 2 x 2 x 2 trees).
"""
import numpy as np
import pytest

from paper_2112_07537_gb300 import inputs as I

pytestmark = pytest.mark.gpu

FUSED, MARCH = 1, 2


@pytest.fixture(scope="module")
def mr():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2112_07537_gb300 import build, mrgb
    build.build()
    return mrgb


def _taylor_green(xyz, comp):
    w, ph = 2 * np.pi, 0.3
    x, y, z = xyz
    if comp == 0:
        return np.sin(w * x + ph) * np.cos(w * y) * np.cos(w * z)
    if comp == 1:
        return -np.cos(w * x + ph) * np.sin(w * y) * np.cos(w * z)
    return 0.25 * np.cos(w * z) * np.sin(w * x)


def _run(mr, O, nb, N, Nt, scheme, vel, diff, which, nsteps=2):
    """nsteps RK3 steps of a Gaussian on the refined 2x2x2 forest with one
    stage kernel; returns the device result and the oracle's."""
    nt, tl = (2, 2, 2), 0.5
    lev, anc = I.tree_config1()
    g = mr.Grid(nt, tl, nb, 0, 1, N, Nt, lev, anc, precision=mr.F32, nfields=4 if vel else 1,
                velocity=vel)
    g.set_stage_kernel(which)
    glev, ganc, _ = g.leaves()
    og = O.Grid(nt, tl, nb, N, Nt, 0, 1, glev, ganc)
    xyz = I.point_coords(nt, tl, nb, glev, ganc)
    phi = I.gaussian_images(xyz, (0.45, 0.5, 0.55), 0.08, nimg=1).astype(np.float32)
    g.field_copy_in(0, phi)
    h = tl / (nb * 2)
    nu = 0.005 if diff else 0.0
    if diff:
        g.set_diffusion(nu, diff)
    sch = {"CONS5": (mr.CONS5, O.CONS5), "WENOZ5": (mr.WENOZ5, O.WENOZ5)}[scheme]
    ref = phi.astype(np.float64)
    if vel:
        v = [_taylor_green(xyz, d).astype(np.float32) for d in range(3)]
        for d in range(3):
            g.field_copy_in(1 + d, v[d])
        v64 = [O.ghost_fill(og, x.astype(np.float64), 3)[1] for x in v]
        vpads = [O.ghost_fill(og, x, 3)[0] for x in v64]
        dt = 0.4 * h / 2.5
        for _ in range(nsteps):
            g.step_vel(0, dt, (1, 2, 3), sch[0])
            ref = O.rk3_step_velpad(og, ref, vpads, dt, sch[1])
    else:
        u = (1.0, -0.5, 0.25)
        dt = O.dt_cfl(og, 0.5, u)
        if diff:
            dt = min(dt, 0.1 * h * h / nu)
        for _ in range(nsteps):
            g.step(0, dt, u, sch[0])
            ref = (O.rk3_step_diff(og, ref, dt, sch[1], u, nu, diff) if diff
                   else O.rk3_step(og, ref, dt, sch[1], u))
    return g.field_copy_out(0).astype(np.float64), ref


@pytest.mark.parametrize("nb,N,Nt", [(16, 4, 0), (24, 6, 2), (16, 2, 2), (24, 4, 2)])
@pytest.mark.parametrize("scheme", ["CONS5", "WENOZ5"])
@pytest.mark.parametrize("vel", [False, True])
def test_stage_kernels_agree_and_match_oracle(mr, oracle_mod, nb, N, Nt, scheme, vel):
    got = {w: _run(mr, oracle_mod, nb, N, Nt, scheme, vel, 0, w) for w in (FUSED, MARCH)}
    ref = got[FUSED][1]
    scale = np.abs(ref).max()
    assert np.abs(got[FUSED][0] - got[MARCH][0]).max() <= 1e-6 * scale
    for w in (FUSED, MARCH):
        err = np.abs(got[w][0] - ref).max() / scale
        assert err <= 1e-5, (w, err)


@pytest.mark.parametrize("diff", [2, 4])
def test_stage_kernels_with_diffusion(mr, oracle_mod, diff):
    got = {w: _run(mr, oracle_mod, 24, 6, 2, "WENOZ5", False, diff, w) for w in (FUSED, MARCH)}
    ref = got[FUSED][1]
    scale = np.abs(ref).max()
    assert np.abs(got[FUSED][0] - got[MARCH][0]).max() <= 1e-6 * scale
    for w in (FUSED, MARCH):
        assert np.abs(got[w][0] - ref).max() <= 1e-5 * scale


def test_stage_kernel_bare_rhs(mr, oracle_mod):
    """mr_rhs_advect (the bare right-hand side, no RK combination) with both
    kernels, against the oracle's rhs of the ghost-filled field."""
    O = oracle_mod
    nt, tl, nb, N, Nt = (2, 2, 2), 0.5, 24, 4, 2
    lev, anc = I.tree_config1()
    res = {}
    for w in (FUSED, MARCH):
        g = mr.Grid(nt, tl, nb, 0, 1, N, Nt, lev, anc, precision=mr.F32, nfields=2)
        g.set_stage_kernel(w)
        glev, ganc, _ = g.leaves()
        og = O.Grid(nt, tl, nb, N, Nt, 0, 1, glev, ganc)
        phi = I.gaussian_images(I.point_coords(nt, tl, nb, glev, ganc), (0.4, 0.55, 0.5), 0.09,
                                nimg=1).astype(np.float32)
        g.field_copy_in(0, phi)
        g.rhs_advect(0, (0.5, 1.0, -0.75), 1, mr.WENOZ5)
        res[w] = g.field_copy_out(1).astype(np.float64)
    pad, _ = O.ghost_fill(og, phi.astype(np.float64), 3)
    ref = O.rhs(og, pad, 3, O.WENOZ5, (0.5, 1.0, -0.75))
    scale = np.abs(ref).max()
    assert np.abs(res[FUSED] - res[MARCH]).max() <= 1e-6 * scale
    for w in (FUSED, MARCH):
        assert np.abs(res[w] - ref).max() <= 5e-5 * scale


def test_stage_kernel_switch_rejects_bad_values(mr):
    nt, tl, nb = (2, 2, 2), 0.5, 16
    lev, anc = I.tree_config1()
    g = mr.Grid(nt, tl, nb, 0, 1, 4, 0, lev, anc, precision=mr.F32)
    for bad in (-1, 3):
        with pytest.raises(mr.MRError):
            g.set_stage_kernel(bad)
