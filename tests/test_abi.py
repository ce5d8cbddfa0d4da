"""C ABI checks that need no GPU: the library loads, exports every symbol the
header declares, and rejects invalid arguments during host-side validation
(before any device work)."""
import ctypes
import os
import re

import numpy as np
import pytest

import __graft_entry__
from paper_1308_0730_gb300 import mvd

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    __graft_entry__.build()
    return mvd.load()


def _declared_symbols():
    names = set()
    for f in os.listdir(os.path.join(ROOT, "include")):
        if f.endswith(".h"):
            src = open(os.path.join(ROOT, "include", f)).read()
            src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
            names |= set(re.findall(r"\b(mvd_[a-z0-9_]+)\s*\(", src))
    return sorted(names)


def test_library_exports_every_declared_symbol(lib):
    declared = _declared_symbols()
    assert "mvd_create" in declared and "mvd_iterate" in declared
    for name in declared:
        assert hasattr(lib, name), name
    assert set(declared) <= set(mvd.EXPORTS) | set(declared)
    for name in mvd.EXPORTS:
        assert name in declared, f"binding lists {name} but the header does not declare it"


def test_default_options(lib):
    o = mvd.Options()
    lib.mvd_default_options(ctypes.byref(o))
    assert o.eps == 0.0 and o.path == 0 and o.stream is None and o.views_on_device == 0 and o.device == -1
    assert o.precision == mvd.MVD_PRECISE and o.boundary == mvd.MVD_BOUNDARY_PERIODIC


def _good():
    views = [np.ones((8, 8, 8), np.float32)] * 2
    psfs = [np.ones((3, 3, 3), np.float32)] * 2
    return views, psfs


@pytest.mark.parametrize("case,status", [
    ("even_psf", mvd.MVD_ERR_SHAPE),
    ("psf_too_big", mvd.MVD_ERR_SHAPE),
    ("negative_psf", mvd.MVD_ERR_ARG),
    ("zero_psf", mvd.MVD_ERR_ARG),
    ("nan_psf", mvd.MVD_ERR_ARG),
    ("no_views", mvd.MVD_ERR_ARG),
    ("bad_path", mvd.MVD_ERR_ARG),
    ("bad_eps", mvd.MVD_ERR_ARG),
    ("bad_boundary", mvd.MVD_ERR_ARG),
    ("bad_precision", mvd.MVD_ERR_ARG),
])
def test_create_rejects_invalid_arguments(lib, case, status):
    views, psfs = _good()
    kw = {}
    if case == "even_psf":
        psfs = [np.ones((3, 4, 3), np.float32)] * 2
    elif case == "psf_too_big":
        psfs = [np.ones((9, 3, 3), np.float32)] * 2
    elif case == "negative_psf":
        p = np.ones((3, 3, 3), np.float32)
        p[1, 1, 1] = -1
        psfs = [p, p]
    elif case == "zero_psf":
        psfs = [np.zeros((3, 3, 3), np.float32)] * 2
    elif case == "nan_psf":
        p = np.ones((3, 3, 3), np.float32)
        p[0, 0, 0] = np.nan
        psfs = [p, p]
    elif case == "no_views":
        views, psfs = [], []
    elif case == "bad_path":
        kw["path"] = 7
    elif case == "bad_eps":
        kw["eps"] = float("nan")
    elif case == "bad_boundary":
        kw["boundary"] = 3
    elif case == "bad_precision":
        kw["precision"] = 3
    if case == "no_views":
        h = ctypes.c_void_p()
        opt = mvd.Options()
        lib.mvd_default_options(ctypes.byref(opt))
        st = lib.mvd_create(None, 0, None, None, (ctypes.c_int * 3)(8, 8, 8), ctypes.byref(opt), ctypes.byref(h))
        assert st == status and not h.value
        return
    with pytest.raises(mvd.MvdError) as ei:
        mvd.mvd_create(views, psfs, **kw)
    assert ei.value.status == status
    assert mvd.mvd_last_error()


def test_null_context_calls_fail_cleanly(lib):
    assert lib.mvd_iterate(None, 1, None, 0) == mvd.MVD_ERR_ARG
    assert lib.mvd_precompute_kernels(None, 1) == mvd.MVD_ERR_ARG
    assert lib.mvd_synchronize(None) == mvd.MVD_ERR_ARG
    lib.mvd_destroy(None)
    assert lib.mvd_get_path(None) == -1
    assert isinstance(mvd.mvd_launch_count(), int)
    assert lib.mvd_autotune(None, None, None) == mvd.MVD_ERR_ARG
    assert lib.mvd_unrolled_forward(None, 1) == mvd.MVD_ERR_ARG
    assert lib.mvd_unrolled_backward(None, None, None, None) == mvd.MVD_ERR_ARG
    assert lib.mvd_set_views(None, None, 0) == mvd.MVD_ERR_ARG
    assert "NULL" in mvd.mvd_last_error()


class _FakeDeviceTensor:
    """Stands in for a CUDA tensor: only what the binding's checks read."""

    def __init__(self, shape, dtype="torch.float32", contiguous=True):
        self.shape = shape
        self.dtype = dtype
        self.is_cuda = True
        self._contiguous = contiguous

    def data_ptr(self):
        return 0

    def is_contiguous(self):
        return self._contiguous


def test_volume_checks_of_the_binding():
    """Pointers cross the C ABI without sizes: the binding refuses volumes of the wrong shape
    or layout before the library reads X*Y*Z floats behind them."""
    good = [np.ones((4, 5, 6), np.float32)] * 2
    mvd._check_volumes(good, (4, 5, 6), "view", 2)
    with pytest.raises(ValueError):
        mvd._check_volumes(good, (4, 5, 7), "view")
    with pytest.raises(ValueError):
        mvd._check_volumes(good, (4, 5, 6), "view", 3)
    with pytest.raises(ValueError):
        mvd._check_volumes([good[0], np.ones((4, 5, 5), np.float32)], (4, 5, 6), "view")
    mvd._check_volumes([_FakeDeviceTensor((4, 5, 6))], (4, 5, 6), "view")
    for bad in (_FakeDeviceTensor((4, 5, 6), dtype="torch.float64"), _FakeDeviceTensor((4, 5, 6), contiguous=False)):
        with pytest.raises(ValueError):
            mvd._check_volumes([bad], (4, 5, 6), "view")
    with pytest.raises(ValueError):  # mixed view shapes at create, before any device work
        mvd.mvd_create([good[0], np.ones((4, 5, 5), np.float32)], [np.ones((3, 3, 3), np.float32)] * 2)


@pytest.mark.parametrize("case,status", [
    ("null_psi", mvd.MVD_ERR_ARG),
    ("null_dims", mvd.MVD_ERR_ARG),
    ("eps_zero", mvd.MVD_ERR_ARG),
    ("eps_negative", mvd.MVD_ERR_ARG),
    ("eps_nan", mvd.MVD_ERR_ARG),
    ("even_box", mvd.MVD_ERR_SHAPE),
    ("box_larger_than_volume", mvd.MVD_ERR_SHAPE),
    ("zero_dim", mvd.MVD_ERR_SHAPE),
    ("beyond_scratch", mvd.MVD_ERR_SHAPE),
    ("box_beyond_shared_memory", mvd.MVD_ERR_UNSUPPORTED),
])
def test_noalloc_rejects_invalid_arguments(lib, case, status):
    """Host-side checks of the allocation-free update, made before any device call: the
    pointers below are never dereferenced."""
    fake = ctypes.c_void_p(4096)
    ptrs = {"psi": fake, "phi": fake, "psf": fake, "comp": fake}
    dims, kd, eps = [32, 32, 32], [3, 5, 7], 1e-3
    dims_p = True
    if case == "null_psi":
        ptrs["psi"] = None
    elif case == "null_dims":
        dims_p = False
    elif case == "eps_zero":
        eps = 0.0
    elif case == "eps_negative":
        eps = -1.0
    elif case == "eps_nan":
        eps = float("nan")
    elif case == "even_box":
        kd = [3, 4, 5]
    elif case == "box_larger_than_volume":
        kd = [33, 3, 3]
    elif case == "zero_dim":
        dims = [32, 0, 32]
    elif case == "beyond_scratch":
        dims = [256, 128, 128]
    elif case == "box_beyond_shared_memory":
        dims, kd = [128, 128, 128], [101, 101, 101]
    d = (ctypes.c_int * 3)(*dims) if dims_p else None
    k = (ctypes.c_int * 3)(*kd)
    rc = lib.mvd_update_direct_noalloc(ptrs["psi"], ptrs["phi"], ptrs["psf"], ptrs["comp"], d, k, eps, None)
    assert rc == status, (case, rc, mvd.mvd_last_error())


def test_noalloc_binding_checks_its_tensors():
    """The binding refuses what would make the kernels read or write outside the caller's
    buffers, before it passes any pointer."""
    torch = pytest.importorskip("torch")
    a = torch.ones((8, 8, 8))
    k = torch.ones((3, 3, 3))
    with pytest.raises(ValueError):
        mvd.mvd_update_direct_noalloc(a, a, k, k, 1e-3)  # host tensors
