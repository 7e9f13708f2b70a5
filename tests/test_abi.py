"""The C-ABI library builds, loads and exports every entry point that
include/mrgb.h declares (no GPU needed: no compute call is made)."""
import ctypes
import os
import re

from conftest import ROOT


def _declared():
    src = open(os.path.join(ROOT, "include", "mrgb.h")).read()
    return sorted(set(re.findall(r"^\s*(?:const\s+)?\w+\s*\*?\s*(mr_\w+)\s*\(", src, re.M)))


def test_library_exports_every_declared_symbol():
    from paper_2112_07537_gb300 import build, mrgb
    path = build.build()
    lib = ctypes.CDLL(path)
    declared = _declared()
    assert len(declared) >= 15
    missing = [s for s in declared if not hasattr(lib, s)]
    assert not missing, missing
    assert sorted(mrgb.EXPORTS) == declared


def test_workspace_size_and_descriptor_validation():
    from paper_2112_07537_gb300 import mrgb
    L = mrgb.load()
    d = mrgb.Desc()
    d.ntree[:] = [2, 2, 2]
    d.tree_len, d.nb, d.lmin, d.lmax = 0.5, 16, 0, 1
    d.wav_N, d.wav_Nt, d.precision, d.nfields, d.capacity = 4, 0, mrgb.F32, 1, 15
    n = ctypes.c_size_t()
    assert L.mr_workspace_size(ctypes.byref(d), ctypes.byref(n)) == 0
    assert n.value > 15 * 16 ** 3 * 4
    d.nb = 15  # odd block size
    assert L.mr_workspace_size(ctypes.byref(d), ctypes.byref(n)) == -1
    d.nb, d.wav_N = 16, 3
    assert L.mr_workspace_size(ctypes.byref(d), ctypes.byref(n)) == -1


def test_set_diffusion_argument_checks():
    """mr_set_diffusion rejects bad arguments before touching a grid (a null
    grid is refused first, so no device is needed)."""
    from paper_2112_07537_gb300 import build, mrgb
    build.build()
    L = mrgb.load()
    assert L.mr_set_diffusion(None, 0.1, 2) == -1  # MR_ERR_INVALID
