"""Python binding of the C ABI in include/mrgb.h (argument marshalling only).

Every numerical step runs in the CUDA library ``_lib/libmrgb.so``; this module
only converts arguments.  PyTorch supplies device memory (the grid workspace
is a torch uint8 tensor) and the stream.  If the library is missing or fails
to load, ``load()`` raises: there is no fallback path.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_lib", "libmrgb.so")

MR_OK = 0
F32, F64 = 0, 1
CONS3, CONS5, WENOZ5 = 0, 1, 2
INIT_GAUSSIAN, INIT_TANH_SPHERE, INIT_TAYLOR_GREEN, INIT_GAUSSIAN_SUM = 0, 1, 2, 3
ADAPT_REFINE, ADAPT_COARSEN = 1, 2
ADAPT_OTHERS_FP64 = 4  # FP32 grids: the non-criterion fields adapt in FP64 arithmetic
INIT_COMPACT_GAUSSIAN, INIT_DEFORMATION, INIT_GAUSSIAN_SUM_ADD = 4, 5, 6
GRID_FIXED_TREE = 1
GRID_VELOCITY = 2
GRID_INDEPENDENT_TREES = 4
GRID_BOUNDED_X, GRID_BOUNDED_Y, GRID_BOUNDED_Z = 8, 16, 32
GRID_BC_DIRICHLET0, GRID_BC_ZERO = 64, 128
BC_EXTRAP, BC_DIRICHLET0, BC_ZERO = 0, 1, 2  # boundary conditions (flag bits above)
NUM_KERNELS = 18

# every entry point include/mrgb.h declares
EXPORTS = ["mr_last_error", "mr_workspace_size", "mr_grid_create", "mr_grid_destroy",
           "mr_grid_leaves", "mr_field_copy_in", "mr_field_copy_out", "mr_field_set",
           "mr_ghost_fill", "mr_ghost_fill64", "mr_sync", "mr_rhs_advect", "mr_rk_stage",
           "mr_step", "mr_criterion", "mr_adapt", "mr_adapt_iter", "mr_mass", "mr_query",
           "mr_field_ptr", "mr_profile", "mr_profile_read", "mr_launch_count", "mr_profile_bytes", "mr_set_diffusion", "mr_step_vel_scaled",
           "mr_ghost_fill_static", "mr_rhs_advect_vel", "mr_step_vel", "mr_velocity_invalidate",
           "mr_device_peaks", "mr_dt", "mr_use_graphs", "mr_graph_replays", "mr_set_adapt_limits",
           "mr_last_block_norms", "mr_autotune", "mr_autotune_table", "mr_autotune_clear",
           "mr_set_stage_kernel"]


class MRError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"mrgb error {code}: {msg}")
        self.code = code


class Desc(C.Structure):
    _fields_ = [("ntree", C.c_int * 3), ("tree_len", C.c_double), ("nb", C.c_int),
                ("lmin", C.c_int), ("lmax", C.c_int), ("wav_N", C.c_int), ("wav_Nt", C.c_int),
                ("precision", C.c_int), ("nfields", C.c_int), ("capacity", C.c_int),
                ("stream", C.c_void_p), ("flags", C.c_int)]


class Stats(C.Structure):
    _fields_ = [("nleaf", C.c_int), ("count_per_level", C.c_int * 32), ("min_level", C.c_int),
                ("max_level", C.c_int)]


_lib = None


def load(path: str = LIB_PATH):
    """Load the CUDA library (raises if it is missing: no CPU fallback)."""
    global _lib
    if _lib is None:
        if not os.path.exists(path):
            raise ImportError(f"CUDA library not built: {path} (run paper_2112_07537_gb300.build)")
        L = C.CDLL(path)
        vp, ip, dp = C.c_void_p, C.POINTER(C.c_int32), C.POINTER(C.c_double)
        L.mr_last_error.restype = C.c_char_p
        L.mr_workspace_size.argtypes = [C.POINTER(Desc), C.POINTER(C.c_size_t)]
        L.mr_grid_create.argtypes = [C.POINTER(Desc), vp, C.c_size_t, ip, ip, C.c_int,
                                     C.POINTER(vp)]
        L.mr_grid_destroy.argtypes = [vp]
        L.mr_grid_leaves.argtypes = [vp, ip, ip, C.POINTER(C.c_uint64), C.c_int,
                                     C.POINTER(C.c_int)]
        L.mr_field_copy_in.argtypes = [vp, C.c_int, vp, C.c_int]
        L.mr_field_copy_out.argtypes = [vp, C.c_int, vp, C.c_int]
        L.mr_field_set.argtypes = [vp, C.c_int, C.c_int, dp, C.c_int]
        L.mr_ghost_fill.argtypes = [vp, C.c_int, C.c_int, vp]
        L.mr_ghost_fill64.argtypes = [vp, C.c_int, C.c_int, vp]
        L.mr_ghost_fill_static.argtypes = [vp, C.c_int, C.c_int, vp]
        L.mr_rhs_advect_vel.argtypes = [vp, C.c_int, ip, C.c_int, C.c_int]
        L.mr_step_vel.argtypes = [vp, C.c_int, C.c_double, ip, C.c_int]
        L.mr_velocity_invalidate.argtypes = [vp]
        L.mr_sync.argtypes = [vp]
        L.mr_rhs_advect.argtypes = [vp, C.c_int, dp, C.c_int, C.c_int]
        L.mr_rk_stage.argtypes = [vp, C.c_int, C.c_double, C.c_int, C.c_int, C.c_int, C.c_int]
        L.mr_step.argtypes = [vp, C.c_int, C.c_double, dp, C.c_int]
        L.mr_criterion.argtypes = [vp, C.c_int, vp]
        L.mr_adapt.argtypes = [vp, C.c_int, C.c_double, C.c_double, C.c_int, C.POINTER(C.c_int)]
        L.mr_adapt_iter.argtypes = [vp, C.c_int, C.c_double, C.c_double, C.c_int,
                                    C.POINTER(C.c_int)]
        L.mr_mass.argtypes = [vp, C.c_int, dp]
        L.mr_query.argtypes = [vp, C.POINTER(Stats)]
        L.mr_field_ptr.argtypes = [vp, C.c_int, C.POINTER(vp)]
        L.mr_profile.argtypes = [vp, C.c_int]
        L.mr_profile_read.argtypes = [vp, C.c_int, dp, C.POINTER(C.c_int), C.POINTER(C.c_char_p)]
        L.mr_profile_bytes.argtypes = [vp, C.c_int, dp]
        L.mr_set_diffusion.argtypes = [vp, C.c_double, C.c_int]
        L.mr_step_vel_scaled.argtypes = [vp, C.c_int, C.c_double, ip, C.c_int, dp]
        L.mr_launch_count.argtypes = [vp, C.POINTER(C.c_longlong)]
        L.mr_device_peaks.argtypes = [dp]
        L.mr_dt.argtypes = [vp, C.c_double, dp, ip, dp]
        L.mr_use_graphs.argtypes = [vp, C.c_int]
        L.mr_graph_replays.argtypes = [vp, C.POINTER(C.c_longlong)]
        L.mr_set_adapt_limits.argtypes = [vp, C.c_int, C.c_int]
        L.mr_last_block_norms.argtypes = [vp, vp, C.c_int, C.POINTER(C.c_int)]
        L.mr_autotune.argtypes = [vp, C.c_int]
        L.mr_set_stage_kernel.argtypes = [vp, C.c_int]
        L.mr_autotune_table.argtypes = [C.c_char_p, C.c_size_t, C.POINTER(C.c_int)]
        _lib = L
    return _lib


PEAK_NAMES = ("fp32_fma_tflops", "fp64_fma_tflops", "fp32_fast_div_gps", "fp32_div_gps",
              "fp64_div_gps")


def device_peaks():
    """Measured compute throughput of the current device (mr_device_peaks)."""
    out = (C.c_double * len(PEAK_NAMES))()
    _chk(load().mr_device_peaks(out))
    return dict(zip(PEAK_NAMES, list(out)))


def autotune_table():
    """Lines of the process-wide autotuner table (one per tuned launch shape)."""
    n = C.c_int()
    buf = C.create_string_buffer(1 << 16)
    _chk(load().mr_autotune_table(buf, len(buf), C.byref(n)))
    return [ln for ln in buf.value.decode().splitlines() if ln]


def autotune_clear():
    _chk(load().mr_autotune_clear())


def _chk(code):
    if code != MR_OK:
        raise MRError(code, load().mr_last_error().decode())
    return code


def _u3(u):
    return (C.c_double * 3)(*[float(v) for v in u])


def _ptr(x):
    """Raw pointer of a torch tensor or numpy array (argument marshalling)."""
    if hasattr(x, "data_ptr"):
        return C.c_void_p(x.data_ptr())
    return C.c_void_p(x.ctypes.data)


def _on_dev(x):
    return int(hasattr(x, "is_cuda") and x.is_cuda)


class Grid:
    """A forest of octrees of nb^3 blocks on one GPU (mr_grid): periodic, or
    with physical boundaries along the axes with bounded[d] = 1 and boundary
    condition bc (BC_EXTRAP, BC_DIRICHLET0 or BC_ZERO)."""

    def __init__(self, ntree, tree_len, nb, lmin, lmax, N, Nt, lev, anc, precision=F32,
                 nfields=1, capacity=None, device="cuda", stream=None, fixed_tree=False,
                 velocity=False, independent_trees=False, bounded=(0, 0, 0), bc=BC_EXTRAP):
        import torch
        L = load()
        lev = np.ascontiguousarray(lev, np.int32)
        anc = np.ascontiguousarray(np.asarray(anc).reshape(-1, 3), np.int32)
        cap = int(capacity or len(lev))
        self.torch = torch
        self.device = torch.device(device)
        s = stream if stream is not None else torch.cuda.current_stream(self.device)
        self.stream = s
        d = Desc()
        d.ntree[:] = list(ntree)
        d.tree_len, d.nb, d.lmin, d.lmax = float(tree_len), nb, lmin, lmax
        d.wav_N, d.wav_Nt, d.precision, d.nfields, d.capacity = N, Nt, precision, nfields, cap
        d.stream = s.cuda_stream
        d.flags = ((GRID_FIXED_TREE if fixed_tree else 0) | (GRID_VELOCITY if velocity else 0) |
                   (GRID_INDEPENDENT_TREES if independent_trees else 0) |
                   sum(f for f, on in zip((GRID_BOUNDED_X, GRID_BOUNDED_Y, GRID_BOUNDED_Z), bounded) if on) |
                   {BC_EXTRAP: 0, BC_DIRICHLET0: GRID_BC_DIRICHLET0, BC_ZERO: GRID_BC_ZERO}[bc])
        self.desc = d
        nbytes = C.c_size_t()
        _chk(L.mr_workspace_size(C.byref(d), C.byref(nbytes)))
        self.ws = torch.empty(nbytes.value + 256, dtype=torch.uint8, device=self.device)
        base = self.ws.data_ptr()
        self._off = (-base) % 256
        h = C.c_void_p()
        _chk(L.mr_grid_create(C.byref(d), C.c_void_p(base + self._off), nbytes.value,
                              lev.ctypes.data_as(C.POINTER(C.c_int32)),
                              anc.ctypes.data_as(C.POINTER(C.c_int32)), len(lev), C.byref(h)))
        self.h = h
        self.nb, self.N, self.Nt = nb, N, Nt
        self.ntree, self.tree_len, self.lmin, self.lmax = tuple(ntree), float(tree_len), lmin, lmax
        self.precision = precision
        self.dtype = torch.float32 if precision == F32 else torch.float64
        self.np_dtype = np.float32 if precision == F32 else np.float64
        self.nfields = nfields

    def __del__(self):
        try:
            if getattr(self, "h", None):
                load().mr_grid_destroy(self.h)
                self.h = None
        except Exception:
            pass

    # ------------------------------------------------------------ queries
    @property
    def nleaf(self):
        n = C.c_int()
        _chk(load().mr_grid_leaves(self.h, None, None, None, 0, C.byref(n)))
        return n.value

    def leaves(self):
        n = self.nleaf
        lev = np.empty(n, np.int32)
        anc = np.empty((n, 3), np.int32)
        keys = np.empty(n, np.uint64)
        nn = C.c_int()
        _chk(load().mr_grid_leaves(self.h, lev.ctypes.data_as(C.POINTER(C.c_int32)),
                                   anc.ctypes.data_as(C.POINTER(C.c_int32)),
                                   keys.ctypes.data_as(C.POINTER(C.c_uint64)), n, C.byref(nn)))
        return lev, anc, keys

    def query(self):
        st = Stats()
        _chk(load().mr_query(self.h, C.byref(st)))
        return st

    def sync(self):
        _chk(load().mr_sync(self.h))

    def field_view(self, fid):
        """Torch view (nleaf, nb, nb, nb) of field fid inside the workspace."""
        p = C.c_void_p()
        _chk(load().mr_field_ptr(self.h, fid, C.byref(p)))
        off = p.value - self.ws.data_ptr()
        n = self.nleaf * self.nb ** 3
        es = 4 if self.precision == F32 else 8
        return self.ws[off:off + n * es].view(self.dtype).view(self.nleaf, self.nb, self.nb, self.nb)

    # ------------------------------------------------------------- fields
    def field_copy_in(self, fid, src):
        if not _on_dev(src):
            src = np.ascontiguousarray(src, self.np_dtype)
        elif src.dtype != self.dtype or not src.is_contiguous():
            raise ValueError("device source must be contiguous and of the grid's dtype")
        _chk(load().mr_field_copy_in(self.h, fid, _ptr(src), _on_dev(src)))
        self._keep = src

    def field_copy_out(self, fid, dst=None):
        if dst is None:
            dst = np.empty((self.nleaf, self.nb, self.nb, self.nb), self.np_dtype)
        _chk(load().mr_field_copy_out(self.h, fid, _ptr(dst), _on_dev(dst)))
        return dst

    def field_set(self, fid, kind, params):
        p = (C.c_double * len(params))(*params)
        _chk(load().mr_field_set(self.h, fid, kind, p, len(params)))

    # ------------------------------------------------------------ the path
    def ghost_fill(self, fid, G, padded=None):
        _chk(load().mr_ghost_fill(self.h, fid, G, _ptr(padded) if padded is not None else None))
        return padded

    def ghost_fill_static(self, fid, G, padded=None):
        """mr_ghost_fill without allocation (static device scratch)."""
        _chk(load().mr_ghost_fill_static(self.h, fid, G, _ptr(padded) if padded is not None else None))
        return padded

    def ghost_fill64(self, fid, G, padded=None):
        _chk(load().mr_ghost_fill64(self.h, fid, G, _ptr(padded) if padded is not None else None))
        return padded

    def rhs_advect(self, phi_fid, u, out_fid, scheme):
        _chk(load().mr_rhs_advect(self.h, phi_fid, _u3(u), out_fid, scheme))

    def rhs_advect_vel(self, phi_fid, vel_fids, out_fid, scheme):
        v = (C.c_int32 * 3)(*vel_fids)
        _chk(load().mr_rhs_advect_vel(self.h, phi_fid, v, out_fid, scheme))

    def step_vel(self, phi_fid, dt, vel_fids, scheme):
        v = (C.c_int32 * 3)(*vel_fids)
        _chk(load().mr_step_vel(self.h, phi_fid, float(dt), v, scheme))

    def step_vel_scaled(self, phi_fid, dt, vel_fids, scheme, stage_scale):
        """RK3 step with the velocity fields times stage_scale[s] in stage s."""
        v = (C.c_int32 * 3)(*vel_fids)
        sc = (C.c_double * 3)(*[float(x) for x in stage_scale])
        _chk(load().mr_step_vel_scaled(self.h, phi_fid, float(dt), v, scheme, sc))

    def velocity_invalidate(self):
        _chk(load().mr_velocity_invalidate(self.h))

    def rk_stage(self, stage, dt, u_fid, y_fid, rhs_fid, out_fid):
        _chk(load().mr_rk_stage(self.h, stage, float(dt), u_fid, y_fid, rhs_fid, out_fid))

    def step(self, phi_fid, dt, u, scheme):
        _chk(load().mr_step(self.h, phi_fid, float(dt), _u3(u), scheme))

    def criterion(self, fid, maxdet):
        _chk(load().mr_criterion(self.h, fid, _ptr(maxdet)))
        return maxdet

    def adapt(self, crit_fid, eps_r, eps_c, flags=ADAPT_REFINE | ADAPT_COARSEN):
        n = C.c_int()
        _chk(load().mr_adapt(self.h, crit_fid, float(eps_r), float(eps_c), flags, C.byref(n)))
        return n.value

    def adapt_iter(self, crit_fid, eps_r, eps_c, flags=ADAPT_REFINE | ADAPT_COARSEN):
        n = C.c_int()
        _chk(load().mr_adapt_iter(self.h, crit_fid, float(eps_r), float(eps_c), flags,
                                  C.byref(n)))
        return n.value

    def profile(self, enable):
        _chk(load().mr_profile(self.h, int(enable)))

    def profile_read(self):
        """{kernel name: (total ms, launches)} of the recorded launches."""
        out = {}
        for kid in range(NUM_KERNELS):
            t, n, name = C.c_double(), C.c_int(), C.c_char_p()
            _chk(load().mr_profile_read(self.h, kid, C.byref(t), C.byref(n), C.byref(name)))
            if n.value:
                out[name.value.decode()] = (t.value, n.value)
        return out

    def set_diffusion(self, nu, order):
        """Add nu * (DIFF-2 or DIFF-4 Laplacian) to the stencil step (order 0: off)."""
        _chk(load().mr_set_diffusion(self.h, float(nu), int(order)))

    def profile_bytes(self, kid=0):
        """Algorithmic bytes of the recorded launches of kernel id kid."""
        b = C.c_double()
        _chk(load().mr_profile_bytes(self.h, kid, C.byref(b)))
        return b.value

    def launch_count(self):
        n = C.c_longlong()
        _chk(load().mr_launch_count(self.h, C.byref(n)))
        return n.value

    def dt(self, cfl, u=None, vel_fids=None):
        """CFL time step from the constant velocity u or the fields vel_fids."""
        out = C.c_double()
        uu = _u3(u) if u is not None else None
        vv = (C.c_int32 * 3)(*vel_fids) if vel_fids is not None else None
        _chk(load().mr_dt(self.h, float(cfl), uu, vv, C.byref(out)))
        return out.value

    def autotune(self, enable=True):
        """Tune launch shapes on this grid's data at first use (mr_autotune)."""
        _chk(load().mr_autotune(self.h, int(enable)))

    def set_stage_kernel(self, which):
        """FP32 stage kernel: 0 tuned/default, 1 k_fused, 2 k_march (mr_set_stage_kernel)."""
        _chk(load().mr_set_stage_kernel(self.h, int(which)))

    def use_graphs(self, enable=True):
        """Capture each RK step into a CUDA graph and replay it while unchanged."""
        _chk(load().mr_use_graphs(self.h, int(enable)))

    def graph_replays(self):
        n = C.c_longlong()
        _chk(load().mr_graph_replays(self.h, C.byref(n)))
        return n.value

    def set_adapt_limits(self, max_iter=64, max_sweeps=256):
        _chk(load().mr_set_adapt_limits(self.h, int(max_iter), int(max_sweeps)))

    def last_block_norms(self):
        """Block norms the last adaptation iteration decided with (numpy)."""
        n = C.c_int()
        _chk(load().mr_last_block_norms(self.h, None, 0, C.byref(n)))
        out = np.empty(n.value)
        _chk(load().mr_last_block_norms(self.h, out.ctypes.data_as(C.c_void_p), n.value, C.byref(n)))
        return out

    def mass(self, fid):
        m = C.c_double()
        _chk(load().mr_mass(self.h, fid, C.byref(m)))
        return m.value

    # ------------------------------------------------- checkpoint / resume
    def checkpoint(self, path):
        """Write the grid's description, its leaves (Morton order, as
        mr_grid_leaves returns them) and every field (mr_field_copy_out) to
        an .npz file.  Launch-shape, diffusion and graph settings are not
        part of the checkpoint.  A restored field counts as freshly written:
        a checkpoint taken after an RK step (which writes the field) resumes
        bit for bit; right after mr_adapt, the restored grid substitutes the
        fields once more at their next ghost fill, which the adapted grid
        skips (the adaptation left them substituted), so values may differ
        by rounding there.  The ghost-filled velocity cache is rebuilt."""
        d = self.desc
        lev, anc, _ = self.leaves()
        fields = np.stack([self.field_copy_out(f) for f in range(self.nfields)])
        np.savez(path, ntree=np.array(self.ntree), tree_len=self.tree_len, nb=self.nb, lmin=self.lmin,
                 lmax=self.lmax, N=self.N, Nt=self.Nt, precision=self.precision, nfields=self.nfields,
                 capacity=d.capacity, flags=d.flags, lev=lev, anc=anc, fields=fields)

    @classmethod
    def restore(cls, path, device="cuda", stream=None, capacity=None):
        """A new grid from a checkpoint: the same leaves in the same slots
        (mr_grid_create orders them as they were) and the same field values
        (mr_field_copy_in), so every later call gives the results the saved
        grid would have given."""
        z = np.load(path)
        flags = int(z["flags"])
        g = cls(tuple(int(x) for x in z["ntree"]), float(z["tree_len"]), int(z["nb"]), int(z["lmin"]),
                int(z["lmax"]), int(z["N"]), int(z["Nt"]), z["lev"], z["anc"], precision=int(z["precision"]),
                nfields=int(z["nfields"]), capacity=capacity or int(z["capacity"]), device=device,
                stream=stream, fixed_tree=bool(flags & GRID_FIXED_TREE), velocity=bool(flags & GRID_VELOCITY),
                independent_trees=bool(flags & GRID_INDEPENDENT_TREES),
                bounded=tuple(int(bool(flags & f)) for f in (GRID_BOUNDED_X, GRID_BOUNDED_Y, GRID_BOUNDED_Z)),
                bc=BC_ZERO if flags & GRID_BC_ZERO else BC_DIRICHLET0 if flags & GRID_BC_DIRICHLET0 else BC_EXTRAP)
        for f in range(g.nfields):
            g.field_copy_in(f, z["fields"][f])
        return g
