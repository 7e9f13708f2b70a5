"""FP64 CPU oracle for the multiresolution stencil path (ctypes front end).

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and
the CPU-baseline leg of ``bench.py`` may import this module.  It shares no
code with the CUDA path: the arithmetic lives in ``mr_oracle.c``, written
step by step from the paper (Gillis & van Rees, arXiv 2112.07537):

* filter bank: Tables SM1 / SM2 (interleaved H^a, G^a, J^s, K^s);
* ghost fill: Alg. SM1 (same-level copy, refinement of the coarse buffer) and
  Alg. SM2 (substitution, eqs 2.23 / 2.27-2.29; coarsening into coarser
  neighbours), Sec. 2.2.2;
* details and block criterion: Sec. 2.2.5, eqs 2.24-2.26, Table 2.2;
* adaptation: Alg. SM3 (status, policy, refine / coarsen, update step eq 2.22);
* right-hand side: Sec. SM "Finite differences" (Tables SM3 / SM4, WENO-Z);
* time stepping: Sec. SM "Time integration" (RK3-TVD).
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
from dataclasses import dataclass

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "mr_oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")

CONS3, CONS5, WENOZ5 = 0, 1, 2
BC_EXTRAP, BC_DIRICHLET0, BC_ZERO = 0, 1, 2
FINER, SAME, COARSER = 1, 0, -1


def build(force: bool = False) -> str:
    """Compile the oracle (plain C, FP64, no FMA contraction)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        subprocess.check_call(["gcc", "-O2", "-fPIC", "-shared", "-ffp-contract=off",
                               "-o", _LIB, _SRC, "-lm"])
    return _LIB


_lib = None


def lib():
    global _lib
    if _lib is None:
        _lib = C.CDLL(build())
        _declare(_lib)
    return _lib


class _Grid(C.Structure):
    _fields_ = [("nt", C.c_int * 3), ("tree_len", C.c_double), ("nb", C.c_int),
                ("N", C.c_int), ("Nt", C.c_int), ("lmin", C.c_int), ("lmax", C.c_int),
                ("nleaf", C.c_int), ("lev", C.POINTER(C.c_int32)),
                ("anc", C.POINTER(C.c_int32)), ("periodic", C.c_int * 3), ("bc", C.c_int)]


_dp = C.POINTER(C.c_double)
_ip = C.POINTER(C.c_int32)


def _declare(L):
    L.og_ghost_fill.argtypes = [C.POINTER(_Grid), _dp, C.c_int, _dp, _dp]
    L.og_rhs.argtypes = [C.POINTER(_Grid), _dp, C.c_int, C.c_int, _dp, _dp, _dp, _dp, _dp]
    L.og_rk3_step.argtypes = [C.POINTER(_Grid), _dp, C.c_double, C.c_int, _dp]
    L.og_laplacian.argtypes = [C.POINTER(_Grid), _dp, C.c_int, C.c_int, _dp]
    L.og_rk3_step_velpad_scaled.argtypes = [C.POINTER(_Grid), _dp, _dp, _dp, _dp, C.c_double, C.c_int, _dp]
    L.og_rk3_step_diff.argtypes = [C.POINTER(_Grid), _dp, C.c_double, C.c_int, _dp, C.c_double, C.c_int]
    L.og_dt.argtypes = [C.POINTER(_Grid), C.c_double, _dp]
    L.og_dt.restype = C.c_double
    L.og_dt_vel.argtypes = [C.POINTER(_Grid), C.c_double, _dp, _dp, _dp]
    L.og_dt_vel.restype = C.c_double
    L.og_moments.argtypes = [C.POINTER(_Grid), _dp, _dp, _dp]
    L.og_criterion.argtypes = [C.POINTER(_Grid), _dp, C.c_int, _dp]
    L.og_detail_reach.argtypes = [C.c_int, C.c_int, C.POINTER(C.c_int), C.POINTER(C.c_int)]
    L.og_adapt_shell.argtypes = [C.c_int, C.c_int]
    L.og_policy.argtypes = [C.POINTER(_Grid), _ip, C.POINTER(C.c_int8)]
    L.og_adapt_iter.argtypes = [C.POINTER(_Grid), _dp, C.c_double, C.c_double, _ip, C.c_int,
                                C.c_int, _ip, _ip, _dp, _ip, C.POINTER(C.c_int), _dp,
                                C.POINTER(C.c_int8)]
    L.og_adapt_iter_fields.argtypes = [C.POINTER(_Grid), C.c_int, C.POINTER(_dp), C.c_double, C.c_double,
                                       _ip, C.c_int, C.c_int, _ip, _ip, C.POINTER(_dp), _ip,
                                       C.POINTER(C.c_int), _dp, C.POINTER(C.c_int8)]
    L.og_filter_taps.argtypes = [C.c_int, C.c_int, C.c_int, C.POINTER(C.c_int), _dp,
                                 C.POINTER(C.c_int)]
    for f in ("og_restrict_1d", "og_detail_1d"):
        getattr(L, f).argtypes = [C.c_int, C.c_int, C.c_int, _dp, _dp]
    L.og_synth_1d.argtypes = [C.c_int, C.c_int, C.c_int, _dp, _dp, _dp]
    L.og_status.argtypes = [C.c_double, C.c_double, C.c_double]
    L.og_rk3_step_vel.argtypes = [C.POINTER(_Grid), _dp, _dp, _dp, _dp, C.c_double, C.c_int]
    L.og_rk3_step_velpad.argtypes = [C.POINTER(_Grid), _dp, _dp, _dp, _dp, C.c_double, C.c_int]
    L.og_weno_beta.argtypes = [_dp, _dp]
    L.og_iface_flux.argtypes = [C.c_int, _dp, C.c_int]
    L.og_iface_flux.restype = C.c_double
    L.og_morton_key.argtypes = [C.c_int] * 5
    L.og_morton_key.restype = C.c_uint64


def _d(a):
    return a.ctypes.data_as(_dp) if a is not None else None


@dataclass
class Grid:
    """A forest of octrees with its leaves: lev[n], anc[n,3]; periodic along
    the axes with periodic[d] = 1, else bounded with boundary condition bc
    (BC_EXTRAP, BC_DIRICHLET0 or BC_ZERO, Sec. 2.4)."""
    nt: tuple
    tree_len: float
    nb: int
    N: int
    Nt: int
    lmin: int
    lmax: int
    lev: np.ndarray
    anc: np.ndarray
    periodic: tuple = (1, 1, 1)
    bc: int = 0

    def __post_init__(self):
        self.lev = np.ascontiguousarray(self.lev, dtype=np.int32)
        self.anc = np.ascontiguousarray(np.asarray(self.anc).reshape(-1, 3), dtype=np.int32)

    @property
    def nleaf(self):
        return int(self.lev.shape[0])

    def c(self):
        s = _Grid()
        s.nt[:] = list(self.nt)
        s.tree_len, s.nb, s.N, s.Nt = self.tree_len, self.nb, self.N, self.Nt
        s.lmin, s.lmax, s.nleaf = self.lmin, self.lmax, self.nleaf
        s.lev = self.lev.ctypes.data_as(_ip)
        s.anc = self.anc.ctypes.data_as(_ip)
        s.periodic[:] = [int(p) for p in self.periodic]
        s.bc = int(self.bc)
        self._keep = s
        return C.byref(s)

    def with_leaves(self, lev, anc):
        return Grid(self.nt, self.tree_len, self.nb, self.N, self.Nt, self.lmin, self.lmax,
                    lev, anc, self.periodic, self.bc)


def _check(e, what):
    if e < 0:
        raise RuntimeError(f"oracle {what} failed with code {e}")
    return e


def ghost_fill(g: Grid, phi: np.ndarray, G: int):
    """Padded blocks (nleaf, W, W, W) [z, y, x] and the substituted field."""
    phi = np.ascontiguousarray(phi, dtype=np.float64).reshape(g.nleaf, -1)
    W = g.nb + 2 * G
    pad = np.empty((g.nleaf, W, W, W))
    out = np.empty_like(phi)
    _check(lib().og_ghost_fill(g.c(), _d(phi), G, _d(pad), _d(out)), "ghost_fill")
    return pad, out.reshape(g.nleaf, g.nb, g.nb, g.nb)


def rhs(g: Grid, pad: np.ndarray, G: int, scheme: int, u=(1.0, 1.0, 1.0), vel=None):
    pad = np.ascontiguousarray(pad, dtype=np.float64)
    out = np.empty((g.nleaf, g.nb, g.nb, g.nb))
    uc = np.asarray(u, dtype=np.float64) if vel is None else None
    vs = [None, None, None] if vel is None else [np.ascontiguousarray(v, np.float64) for v in vel]
    _check(lib().og_rhs(g.c(), _d(pad), G, scheme, _d(uc), _d(vs[0]), _d(vs[1]), _d(vs[2]),
                        _d(out)), "rhs")
    return out


def laplacian(g: Grid, pad: np.ndarray, G: int, order: int):
    """DIFF-2 / DIFF-4 central Laplacian of a padded field (shell G)."""
    pad = np.ascontiguousarray(pad, dtype=np.float64)
    out = np.empty((g.nleaf, g.nb, g.nb, g.nb))
    _check(lib().og_laplacian(g.c(), _d(pad), G, order, _d(out)), "laplacian")
    return out


def rk3_step_diff(g: Grid, phi: np.ndarray, dt: float, scheme: int, u, nu: float, order: int):
    """RK3 step of d phi/dt = -div(u phi) + nu Laplacian(phi), constant u."""
    phi = np.ascontiguousarray(phi, dtype=np.float64).copy()
    uc = np.asarray(u, dtype=np.float64)
    _check(lib().og_rk3_step_diff(g.c(), _d(phi), dt, scheme, _d(uc), float(nu), int(order)), "rk3_step_diff")
    return phi.reshape(g.nleaf, g.nb, g.nb, g.nb)


def rk3_step(g: Grid, phi: np.ndarray, dt: float, scheme: int, u=(1.0, 1.0, 1.0)):
    phi = np.ascontiguousarray(phi, dtype=np.float64).copy()
    uc = np.asarray(u, dtype=np.float64)
    _check(lib().og_rk3_step(g.c(), _d(phi), dt, scheme, _d(uc)), "rk3_step")
    return phi.reshape(g.nleaf, g.nb, g.nb, g.nb)


def rk3_step_vel(g: Grid, phi: np.ndarray, vel, dt: float, scheme: int):
    """RK3 step with velocity fields (each stage ghost-fills phi and u, v, w);
    returns (phi, vel) -- the velocity components come back substituted."""
    phi = np.ascontiguousarray(phi, dtype=np.float64).copy()
    vs = [np.ascontiguousarray(v, dtype=np.float64).copy() for v in vel]
    _check(lib().og_rk3_step_vel(g.c(), _d(phi), _d(vs[0]), _d(vs[1]), _d(vs[2]), dt, scheme),
           "rk3_step_vel")
    shp = (g.nleaf, g.nb, g.nb, g.nb)
    return phi.reshape(shp), [v.reshape(shp) for v in vs]


def rk3_step_velpad(g: Grid, phi: np.ndarray, vpads, dt: float, scheme: int):
    """RK3 step with the velocity's padded blocks (shell 3) held fixed."""
    phi = np.ascontiguousarray(phi, dtype=np.float64).copy()
    vp = [np.ascontiguousarray(v, dtype=np.float64) for v in vpads]
    _check(lib().og_rk3_step_velpad(g.c(), _d(phi), _d(vp[0]), _d(vp[1]), _d(vp[2]), dt, scheme),
           "rk3_step_velpad")
    return phi.reshape(g.nleaf, g.nb, g.nb, g.nb)


def rk3_step_velpad_scaled(g: Grid, phi: np.ndarray, vpads, dt: float, scheme: int, scale):
    """RK3 step with the fixed padded velocities times scale[s] in stage s."""
    phi = np.ascontiguousarray(phi, dtype=np.float64).copy()
    vp = [np.ascontiguousarray(v, dtype=np.float64) for v in vpads]
    sc = np.asarray(scale, dtype=np.float64)
    _check(lib().og_rk3_step_velpad_scaled(g.c(), _d(phi), _d(vp[0]), _d(vp[1]), _d(vp[2]), dt, scheme,
                                           _d(sc)), "rk3_step_velpad_scaled")
    return phi.reshape(g.nleaf, g.nb, g.nb, g.nb)


def dt_cfl(g: Grid, cfl: float, u) -> float:
    return lib().og_dt(g.c(), cfl, _d(np.asarray(u, dtype=np.float64)))


def dt_cfl_vel(g: Grid, cfl: float, vel) -> float:
    """CFL time step from velocity fields (max over points of sum |u_d|)."""
    v = [np.ascontiguousarray(a, np.float64) for a in vel]
    return lib().og_dt_vel(g.c(), cfl, _d(v[0]), _d(v[1]), _d(v[2]))


def moments(g: Grid, phi: np.ndarray):
    phi = np.ascontiguousarray(phi, dtype=np.float64)
    m0 = C.c_double()
    m1 = np.zeros(3)
    lib().og_moments(g.c(), _d(phi), C.byref(m0), _d(m1))
    return m0.value, m1


def detail_reach(N: int, Nt: int):
    f, b = C.c_int(), C.c_int()
    lib().og_detail_reach(N, Nt, C.byref(f), C.byref(b))
    return f.value, b.value


def adapt_shell(N: int, Nt: int) -> int:
    return lib().og_adapt_shell(N, Nt)


def criterion(g: Grid, pad: np.ndarray, G: int):
    out = np.empty(g.nleaf)
    _check(lib().og_criterion(g.c(), _d(np.ascontiguousarray(pad, np.float64)), G, _d(out)),
           "criterion")
    return out


def block_maxdet(g: Grid, phi: np.ndarray):
    """Ghost fill with the criterion shell, then the per-block max |gamma|."""
    G = adapt_shell(g.N, g.Nt)
    pad, _ = ghost_fill(g, phi, G)
    return criterion(g, pad, G)


def policy(g: Grid, status: np.ndarray, refined=None):
    st = np.ascontiguousarray(status, dtype=np.int8).copy()
    ref = np.zeros(g.nleaf, np.int32) if refined is None else np.ascontiguousarray(refined, np.int32)
    _check(lib().og_policy(g.c(), ref.ctypes.data_as(_ip), st.ctypes.data_as(C.POINTER(C.c_int8))),
           "policy")
    return st


def adapt_iter(g: Grid, phi, eps_r, eps_c, refined=None, allow_refine=True,
               allow_coarsen=True):
    """One iteration of Alg. SM3.  Returns (grid, phi, refined, n_changed,
    maxdet, status) -- maxdet/status on the input grid."""
    phi = np.ascontiguousarray(phi, dtype=np.float64).reshape(g.nleaf, -1)
    ref = np.zeros(g.nleaf, np.int32) if refined is None else np.ascontiguousarray(refined, np.int32)
    cap = 8 * g.nleaf
    lev = np.empty(cap, np.int32)
    anc = np.empty((cap, 3), np.int32)
    out = np.empty((cap, g.nb ** 3))
    rout = np.empty(cap, np.int32)
    md = np.empty(g.nleaf)
    st = np.empty(g.nleaf, np.int8)
    nch = C.c_int()
    flags = (1 if allow_refine else 0) | (2 if allow_coarsen else 0)
    n = _check(lib().og_adapt_iter(g.c(), _d(phi), eps_r, eps_c, ref.ctypes.data_as(_ip), flags,
                                   cap, lev.ctypes.data_as(_ip), anc.ctypes.data_as(_ip),
                                   _d(out), rout.ctypes.data_as(_ip), C.byref(nch), _d(md),
                                   st.ctypes.data_as(C.POINTER(C.c_int8))), "adapt_iter")
    g2 = g.with_leaves(lev[:n].copy(), anc[:n].copy())
    return (g2, out[:n].reshape(n, g.nb, g.nb, g.nb).copy(), rout[:n].copy(), nch.value, md, st)


def adapt_iter_fields(g: Grid, phis, eps_r, eps_c, refined=None, allow_refine=True,
                      allow_coarsen=True):
    """One iteration of Alg. SM3 on several fields; field 0 drives the
    criterion, every field is refined / coarsened / updated.  Returns
    (grid, [fields], refined, n_changed, maxdet, status)."""
    ins = [np.ascontiguousarray(p, dtype=np.float64).reshape(g.nleaf, -1) for p in phis]
    nf = len(ins)
    ref = np.zeros(g.nleaf, np.int32) if refined is None else np.ascontiguousarray(refined, np.int32)
    cap = 8 * g.nleaf
    lev = np.empty(cap, np.int32)
    anc = np.empty((cap, 3), np.int32)
    outs = [np.empty((cap, g.nb ** 3)) for _ in range(nf)]
    rout = np.empty(cap, np.int32)
    md = np.empty(g.nleaf)
    st = np.empty(g.nleaf, np.int8)
    nch = C.c_int()
    pin = (_dp * nf)(*[_d(a) for a in ins])
    pout = (_dp * nf)(*[_d(a) for a in outs])
    flags = (1 if allow_refine else 0) | (2 if allow_coarsen else 0)
    n = _check(lib().og_adapt_iter_fields(g.c(), nf, pin, eps_r, eps_c, ref.ctypes.data_as(_ip), flags, cap,
                                          lev.ctypes.data_as(_ip), anc.ctypes.data_as(_ip), pout,
                                          rout.ctypes.data_as(_ip), C.byref(nch), _d(md),
                                          st.ctypes.data_as(C.POINTER(C.c_int8))), "adapt_iter_fields")
    g2 = g.with_leaves(lev[:n].copy(), anc[:n].copy())
    return (g2, [o[:n].reshape(n, g.nb, g.nb, g.nb).copy() for o in outs], rout[:n].copy(), nch.value,
            md, st)


def adapt(g: Grid, phi, eps_r, eps_c, max_iter=64, **kw):
    """Alg. SM3 to convergence (no block changes)."""
    ref = None
    it = 0
    for it in range(max_iter):
        g, phi, ref, nch, _, _ = adapt_iter(g, phi, eps_r, eps_c, ref, **kw)
        if nch == 0:
            break
    return g, phi, it + 1


def filter_taps(N: int, Nt: int, which: str):
    """Taps of one filter (Ha, Ga, Js, Ks) as (offsets, coefficients)."""
    hw = C.c_int()
    c = np.zeros(13)
    ext = (C.c_int * 2)()
    _check(lib().og_filter_taps(N, Nt, "Ha Ga Js Ks".split().index(which), C.byref(hw), _d(c),
                                ext), "filter_taps")
    h = hw.value
    return np.arange(-h, h + 1), c[:2 * h + 1].copy(), (ext[0], ext[1])


def restrict_1d(N, Nt, fine):
    fine = np.ascontiguousarray(fine, np.float64)
    out = np.empty(fine.size // 2)
    _check(lib().og_restrict_1d(N, Nt, out.size, _d(fine), _d(out)), "restrict_1d")
    return out


def detail_1d(N, Nt, fine):
    fine = np.ascontiguousarray(fine, np.float64)
    out = np.empty(fine.size // 2)
    _check(lib().og_detail_1d(N, Nt, out.size, _d(fine), _d(out)), "detail_1d")
    return out


def synth_1d(N, Nt, lam, gam=None):
    lam = np.ascontiguousarray(lam, np.float64)
    gm = None if gam is None else np.ascontiguousarray(gam, np.float64)
    out = np.empty(2 * lam.size)
    _check(lib().og_synth_1d(N, Nt, lam.size, _d(lam), _d(gm), _d(out)), "synth_1d")
    return out


def weno_beta(v):
    """Smoothness indicators (Table SM4) of the sub-stencils of 5 values."""
    v = np.ascontiguousarray(v, np.float64)
    out = np.empty(3)
    lib().og_weno_beta(_d(v), _d(out))
    return out


def iface_flux(scheme, f6, upwind_left):
    """Interface flux F_{i+1/2} from the point fluxes f_{i-2..i+3}."""
    f6 = np.ascontiguousarray(f6, np.float64)
    return lib().og_iface_flux(int(scheme), _d(f6), int(bool(upwind_left)))


def status(maxdet, eps_r, eps_c):
    return lib().og_status(maxdet, eps_r, eps_c)


def morton_key(lev, ax, ay, az, kl):
    return int(lib().og_morton_key(int(lev), int(ax), int(ay), int(az), int(kl)))
