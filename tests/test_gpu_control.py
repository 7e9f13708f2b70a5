"""Device-side control of the step through the C ABI: the CFL time step
reduced on the device (Sec. 5.1) against the oracle, CUDA-graph replay of RK
steps against stream-ordered steps, and the adaptation's failure paths
(iteration and sweep caps, leaf capacity) raised on the host side of the
library without any device fault."""
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


def _tg(xyz, comp, s=1.0, ph=0.3):
    w = 2 * np.pi
    x, y, z = xyz
    if comp == 0:
        return s * np.sin(w * x + ph) * np.cos(w * y) * np.cos(w * z)
    if comp == 1:
        return -s * np.cos(w * x + ph) * np.sin(w * y) * np.cos(w * z)
    return 0.3 * np.sin(w * z)


@pytest.mark.parametrize("prec", [1, 0])
def test_dt_matches_oracle(mr, oracle_mod, prec):
    """dt = CFL h_min / max sum_d |u_d| (reading of Sec. 5.1) from a constant
    velocity and from velocity fields: the device reduction equals the
    oracle's bit for bit (a maximum is exact; both sides sum the three
    FP64 magnitudes in the same order)."""
    O = oracle_mod
    nt, tl, nb = (2, 2, 2), 0.5, 16
    lev, anc = I.tree_config1()
    g = mr.Grid(nt, tl, nb, 0, 1, 4, 2, lev, anc, precision=prec, nfields=4)
    glev, ganc, _ = g.leaves()
    og = O.Grid(nt, tl, nb, 4, 2, 0, 1, glev, ganc)
    xyz = I.point_coords(nt, tl, nb, glev, ganc)
    vel = [_tg(xyz, d) for d in range(3)]
    if prec == 0:
        vel = [v.astype(np.float32) for v in vel]
    for d in range(3):
        g.field_copy_in(1 + d, vel[d])
    assert g.dt(0.5, u=(1.0, -0.5, 0.25)) == O.dt_cfl(og, 0.5, (1.0, -0.5, 0.25))
    ref = O.dt_cfl_vel(og, 0.5, [v.astype(np.float64) for v in vel])
    assert g.dt(0.5, vel_fids=(1, 2, 3)) == ref
    assert g.dt(0.5, u=(0.0, 0.0, 0.0)) == np.inf
    with pytest.raises(mr.MRError):
        g.dt(-1.0, u=(1.0, 0.0, 0.0))


@pytest.mark.parametrize("prec", [0, 1])
def test_graph_replay_matches_stream_steps(mr, prec):
    """mr_use_graphs: each RK step with velocity fields is captured once and
    replayed; the replayed steps give the same bits as stream-ordered steps,
    a new dt captures again, and constant-velocity steps replay as well."""
    nt, tl, nb = (2, 2, 2), 0.5, 16
    lev, anc = I.tree_config1()
    grids = [mr.Grid(nt, tl, nb, 0, 1, 4, 2, lev, anc, precision=prec, nfields=4, velocity=True)
             for _ in range(2)]
    glev, ganc, _ = grids[0].leaves()
    xyz = I.point_coords(nt, tl, nb, glev, ganc)
    dtype = np.float32 if prec == 0 else np.float64
    phi = I.gaussian(xyz, (0.45, 0.5, 0.55), 0.1).astype(dtype)
    for g in grids:
        g.field_copy_in(0, phi)
        for d in range(3):
            g.field_copy_in(1 + d, _tg(xyz, d).astype(dtype))
    grids[1].use_graphs(True)
    dts = [2e-3, 2e-3, 2e-3, 1.5e-3, 1.5e-3]
    for dt in dts:
        for g in grids:
            g.step_vel(0, dt, (1, 2, 3), mr.WENOZ5)
    assert np.array_equal(grids[0].field_copy_out(0), grids[1].field_copy_out(0))
    assert grids[1].graph_replays() == 3  # captures at the 1st and 4th step
    assert grids[1].launch_count() > grids[0].launch_count() * 0.5
    for _ in range(3):
        for g in grids:
            g.step(0, 1e-3, (1.0, -0.5, 0.25), mr.CONS5)
    assert np.array_equal(grids[0].field_copy_out(0), grids[1].field_copy_out(0))
    assert grids[1].graph_replays() == 5
    grids[1].use_graphs(False)


def _blob_grid(mr, cap):
    nt, tl, nb = (2, 2, 2), 0.5, 16
    lev, anc = I.tree_config1()
    g = mr.Grid(nt, tl, nb, 0, 3, 4, 2, lev, anc, precision=mr.F64, capacity=cap)
    glev, ganc, _ = g.leaves()
    xyz = I.point_coords(nt, tl, nb, glev, ganc)
    # a sharp blob inside the level-1 leaf (1,1,1) of tree 0: it refines, and
    # the policy raises the level-0 roots next to it (2:1)
    g.field_copy_in(0, I.gaussian(xyz, (0.4, 0.4, 0.4), 0.02))
    return g


def test_adaptation_iteration_and_sweep_caps(mr):
    """An adaptation that needs several iterations (a sharp blob refining from
    level 0 to 3) stopped after one returns MR_ERR_TIMEOUT with a consistent
    grid; so does a policy limited to one sweep when a second is needed."""
    g = _blob_grid(mr, 4000)
    g.set_adapt_limits(1, 256)
    with pytest.raises(mr.MRError) as e:
        g.adapt(0, 1e-4, 1e-8)
    assert e.value.code == -4
    lev, anc, keys = g.leaves()
    assert len(lev) > 15 and np.all(np.diff(keys.astype(np.float64)) > 0)
    g.sync()
    g.set_adapt_limits(64, 256)
    assert g.adapt(0, 1e-4, 1e-8) > 0
    g2 = _blob_grid(mr, 4000)
    g2.set_adapt_limits(64, 1)
    with pytest.raises(mr.MRError) as e:
        g2.adapt(0, 1e-4, 1e-8)
    assert e.value.code == -4
    with pytest.raises(mr.MRError):
        g2.set_adapt_limits(0, 1)


def test_adaptation_beyond_capacity_is_refused(mr):
    """Refinement that would exceed the grid's leaf capacity returns
    MR_ERR_NOMEM before any leaf changes; the grid stays usable."""
    g = _blob_grid(mr, 18)  # 15 leaves; one refinement adds 7
    before = g.leaves()
    with pytest.raises(mr.MRError) as e:
        g.adapt_iter(0, 1e-4, 1e-8)
    assert e.value.code == -2
    after = g.leaves()
    assert all(np.array_equal(a, b) for a, b in zip(before, after))
    g.sync()
    g.step(0, 1e-3, (1.0, 0.0, 0.0), mr.CONS5)
    g.sync()


@pytest.mark.parametrize("prec", [0, 1])
def test_autotuned_launches_give_identical_results(mr, prec):
    """The autotuner changes launch shapes only: ghost fills, RK steps with
    velocity fields and an adaptation on a tuning grid equal those of an
    untuned twin -- bit for bit, except that on FP32 grids the tuner also
    picks the faster of the two stage kernels, which evaluate the same
    operations in the same order but may round a multiply-add differently
    where the compiler fuses it (fields within 1e-6 of their maximum) --
    and the table lists the tuned shapes."""
    import torch
    mr.autotune_clear()
    nt, tl, nb = (2, 2, 2), 0.5, 16
    lev, anc = I.tree_config1()
    grids = [mr.Grid(nt, tl, nb, 0, 2, 4, 2, lev, anc, precision=prec, nfields=4, velocity=True,
                     capacity=4000) for _ in range(2)]
    glev, ganc, _ = grids[0].leaves()
    xyz = I.point_coords(nt, tl, nb, glev, ganc)
    dtype = np.float32 if prec == 0 else np.float64
    phi = I.gaussian(xyz, (0.4, 0.4, 0.4), 0.04).astype(dtype)
    for g in grids:
        g.field_copy_in(0, phi)
        for d in range(3):
            g.field_copy_in(1 + d, _tg(xyz, d).astype(dtype))
    # the untuned grid runs first: the table is still empty, so it uses the
    # default shapes; then the tuning grid fills the table
    W = nb + 6
    pads = []
    for k, g in enumerate(grids):
        if k == 1:
            g.autotune(True)
        pad = torch.empty((g.nleaf, W, W, W), dtype=torch.float32 if prec == 0 else torch.float64,
                          device="cuda")
        g.ghost_fill(0, 3, pad)
        for _ in range(2):
            g.step_vel(0, 1e-3, (1, 2, 3), mr.WENOZ5)
        g.adapt(0, 1e-3, 1e-6)
        g.sync()
        pads.append(pad.cpu().numpy())
    assert np.array_equal(pads[0], pads[1])
    assert np.array_equal(grids[0].leaves()[0], grids[1].leaves()[0])
    for f in range(4):
        a, b = grids[0].field_copy_out(f), grids[1].field_copy_out(f)
        if prec == 1:
            assert np.array_equal(a, b)
        else:
            assert np.abs(a.astype(np.float64) - b).max() <= 1e-6 * np.abs(a).max()
    table = mr.autotune_table()
    assert len(table) >= 4, table
    assert any(ln.startswith("k_criterion") for ln in table) and any(ln.startswith("k_prep") for ln in table)
    if prec == 0:  # the FP32 stage kernel (FP64 grids use the plain per-block stage)
        assert any(ln.startswith("k_fused") for ln in table)
        assert any(ln.startswith("stage kernel") for ln in table)


def test_substituted_field_tracking(mr):
    """After a converged mr_adapt every field holds the values the
    adaptation's ghost fill leaves for the current tree; the velocity-cache
    rebuild fills such a component once without writing it back, instead of
    substituting it again (in FP32) first.  A twin grid whose velocity
    fields count as written (mr_field_ptr) before every adaptation gives the
    same bits (the adaptation does not depend on that state); one whose
    fields count as written after the adaptation too takes the two-fill
    cache, and its steps agree within FP32 rounding."""
    nt, tl, nb = (2, 2, 2), 0.5, 16
    lev, anc = I.tree_config1()
    grids = [mr.Grid(nt, tl, nb, 0, 2, 4, 2, lev, anc, precision=mr.F32, nfields=4, velocity=True,
                     capacity=4000) for _ in range(3)]
    glev, ganc, _ = grids[0].leaves()
    xyz = I.point_coords(nt, tl, nb, glev, ganc)
    phi = I.gaussian(xyz, (0.4, 0.4, 0.4), 0.05).astype(np.float32)
    for g in grids:
        g.field_copy_in(0, phi)
        for d in range(3):
            g.field_copy_in(1 + d, _tg(xyz, d).astype(np.float32))
    for cycle in range(3):
        active = grids if cycle == 0 else grids[:2]
        for k, g in enumerate(active):
            if k >= 1:
                for f in range(1, 4):
                    g.field_view(f)  # hands out the pointer: the field counts as written
            g.adapt(0, 1e-3, 1e-6)
        # the adaptation does not depend on that state: bit for bit
        a, b = grids[0].leaves(), grids[1].leaves()
        assert np.array_equal(a[0], b[0]) and np.array_equal(a[1], b[1])
        for f in range(4):
            assert np.array_equal(grids[0].field_copy_out(f), grids[1].field_copy_out(f)), (cycle, f)
        if cycle == 0:
            for f in range(1, 4):
                grids[2].field_view(f)  # the cache of grid 2 takes the two-fill path
        for g in active:
            for _ in range(2):
                g.step_vel(0, 2e-3, (1, 2, 3), mr.WENOZ5)
        assert np.array_equal(grids[1].field_copy_out(0), grids[0].field_copy_out(0))
        if cycle == 0:  # same tree, velocity ghosts differing by FP32 rounding
            ref = grids[0].field_copy_out(0).astype(np.float64)
            other = grids[2].field_copy_out(0).astype(np.float64)
            assert np.abs(other - ref).max() <= 1e-6 * np.abs(ref).max()


def test_checkpoint_restore_resumes_bit_for_bit(mr, tmp_path):
    """Checkpoint / resume: a grid restored from a checkpoint taken after an
    adaptation and two RK3 steps continues exactly like the original (two
    more steps and one more adaptation: same leaves, same field)."""
    nt, tl, nb = (2, 2, 2), 0.5, 16
    lev, anc = I.tree_config1()
    g = mr.Grid(nt, tl, nb, 0, 2, 4, 2, lev, anc, precision=mr.F32, capacity=4000)
    glev, ganc, _ = g.leaves()
    xyz = I.point_coords(nt, tl, nb, glev, ganc)
    g.field_copy_in(0, I.gaussian(xyz, (0.4, 0.4, 0.4), 0.04).astype(np.float32))
    u = (1.0, 0.5, 0.25)
    g.adapt(0, 1e-3, 1e-6)
    for _ in range(2):
        g.step(0, 1e-3, u, mr.WENOZ5)
    path = tmp_path / "grid.npz"
    g.checkpoint(path)
    h = mr.Grid.restore(path)
    assert np.array_equal(h.leaves()[2], g.leaves()[2])
    assert np.array_equal(h.field_copy_out(0), g.field_copy_out(0))
    for x in (g, h):
        for _ in range(2):
            x.step(0, 1e-3, u, mr.WENOZ5)
        x.adapt(0, 1e-3, 1e-6)
    assert np.array_equal(h.leaves()[2], g.leaves()[2])
    assert np.array_equal(h.field_copy_out(0), g.field_copy_out(0))
