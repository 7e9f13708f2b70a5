"""Batches of independent grids (MR_GRID_INDEPENDENT_TREES): every tree of
the forest is its own periodic domain, and all of them advance with one
launch per phase.  Each tree must compute exactly -- bit for bit -- what a
separate one-tree grid with the same leaves and values computes (ghost
fills, RK steps with velocity fields, adaptation), and one tree is checked
against the oracle as well."""
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


def _instance(k):
    """Seeded one-tree grid k: uniform level 1, some leaves refined, 2:1
    balanced within the tree (periodic onto itself)."""
    rng = np.random.default_rng(40 + k)
    lev, anc = I.uniform_leaves((1, 1, 1), 1)
    lev, anc = I.refine_leaves(lev, anc, rng.random(len(lev)) < 0.3 + 0.1 * k)
    return I.balance((1, 1, 1), lev, anc)


def _fields(k, xyz):
    rng = np.random.default_rng(70 + k)
    c = rng.uniform(0.3, 0.7, 3)
    phi = I.gaussian(xyz, tuple(c), 0.06 + 0.02 * k)
    u = rng.normal(size=3)
    u /= np.linalg.norm(u)
    return phi, [np.full_like(phi, u[d]) for d in range(3)]


def _key(lev, anc):
    return [(int(l), tuple(int(x) for x in a)) for l, a in zip(lev, anc)]


@pytest.mark.parametrize("prec", [0, 1])
def test_batched_trees_equal_separate_grids(mr, oracle_mod, prec):
    import torch
    K, nt, tl, nb = 4, (2, 2, 1), 1.0, 16
    dtype = np.float32 if prec == 0 else np.float64
    inst = [_instance(k) for k in range(K)]
    lev, anc, tree = I.batch_leaves(inst, nt)
    batch = mr.Grid(nt, tl, nb, 0, 3, 4, 2, lev, anc, precision=prec, nfields=4, velocity=True,
                    capacity=6000, independent_trees=True)
    singles = [mr.Grid((1, 1, 1), tl, nb, 0, 3, 4, 2, l, a, precision=prec, nfields=4, velocity=True,
                       capacity=2000) for l, a in inst]
    blev, banc, _ = batch.leaves()
    btree = (banc[:, 0] >> blev) % nt[0] + nt[0] * ((banc[:, 1] >> blev) % nt[1])
    bloc = banc - np.stack([(btree % nt[0]), (btree // nt[0]) % nt[1], np.zeros_like(btree)], 1) * \
        (1 << blev)[:, None]
    # the same fields, in every tree's own coordinates
    bf = [np.empty((len(blev), nb, nb, nb), dtype) for _ in range(4)]
    for k, g in enumerate(singles):
        sl, sa, _ = g.leaves()
        xyz = I.point_coords((1, 1, 1), tl, nb, sl, sa)
        phi, vel = _fields(k, xyz)
        vals = [phi] + vel
        for f in range(4):
            g.field_copy_in(f, vals[f].astype(dtype))
        pos = {key: i for i, key in enumerate(_key(sl, sa))}
        for i in np.nonzero(btree == k)[0]:
            j = pos[(int(blev[i]), tuple(int(x) for x in bloc[i]))]
            for f in range(4):
                bf[f][i] = vals[f][j]
    for f in range(4):
        batch.field_copy_in(f, bf[f])

    def compare(tag):
        blev, banc, _ = batch.leaves()
        btree = (banc[:, 0] >> blev) % nt[0] + nt[0] * ((banc[:, 1] >> blev) % nt[1])
        bloc = banc - np.stack([(btree % nt[0]), (btree // nt[0]) % nt[1], np.zeros_like(btree)], 1) * \
            (1 << blev)[:, None]
        outs = [batch.field_copy_out(f) for f in range(4)]
        for k, g in enumerate(singles):
            sl, sa, _ = g.leaves()
            sel = np.nonzero(btree == k)[0]
            assert sorted(_key(blev[sel], bloc[sel])) == sorted(_key(sl, sa)), (tag, k)
            pos = {key: i for i, key in enumerate(_key(sl, sa))}
            for f in range(4):
                so = g.field_copy_out(f)
                for i in sel:
                    j = pos[(int(blev[i]), tuple(int(x) for x in bloc[i]))]
                    assert np.array_equal(outs[f][i], so[j]), (tag, k, f)

    # a ghost fill of every field
    W = nb + 6
    pads = torch.empty((len(blev), W, W, W), dtype=torch.float32 if prec == 0 else torch.float64, device="cuda")
    batch.ghost_fill(0, 3, pads)
    for g in singles:
        g.ghost_fill(0, 3)
    compare("ghost")
    for _ in range(2):
        batch.step_vel(0, 2e-3, (1, 2, 3), mr.WENOZ5)
        for g in singles:
            g.step_vel(0, 2e-3, (1, 2, 3), mr.WENOZ5)
    compare("steps")
    nb_ = batch.adapt(0, 1e-3, 1e-6)
    ns = sum(g.adapt(0, 1e-3, 1e-6) for g in singles)
    assert nb_ == ns and ns > 0
    compare("adapt")
    batch.step_vel(0, 2e-3, (1, 2, 3), mr.WENOZ5)
    for g in singles:
        g.step_vel(0, 2e-3, (1, 2, 3), mr.WENOZ5)
    compare("step after adapt")
    # one tree against the oracle: a ghost fill of the initial field
    if prec == 1:
        O = oracle_mod
        l0, a0 = inst[0]
        og = O.Grid((1, 1, 1), tl, nb, 4, 2, 0, 3, l0, a0)
        g = mr.Grid((1, 1, 1), tl, nb, 0, 3, 4, 2, l0, a0, precision=mr.F64)
        gl, ga, _ = g.leaves()
        og = og.with_leaves(gl, ga)
        phi, _ = _fields(0, I.point_coords((1, 1, 1), tl, nb, gl, ga))
        g.field_copy_in(0, phi)
        pad = torch.empty((len(gl), W, W, W), dtype=torch.float64, device="cuda")
        g.ghost_fill(0, 3, pad)
        ref, _ = O.ghost_fill(og, phi, 3)
        assert np.abs(pad.cpu().numpy() - ref).max() <= 1e-12 * np.abs(phi).max()
