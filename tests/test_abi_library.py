"""Host-side checks of the C ABI library (no GPU needed): it builds for
sm_103a, loads, and exports every function include/gbremd.h declares; the
binding's ctypes structures match the header's field lists."""
import ctypes
import re
import shutil

import pytest

import paper_1803_09652_gb300 as pkg
from paper_1803_09652_gb300 import build as pkg_build


@pytest.fixture(scope="module")
def lib():
    if shutil.which("nvcc") is None and not __import__("os").path.exists("/usr/local/cuda/bin/nvcc"):
        pytest.skip("nvcc not available")
    pkg_build.build()
    return ctypes.CDLL(pkg.LIB_PATH)


def test_header_declares_the_four_hot_path_calls():
    names = pkg.exported_names()
    for n in ("gb_born_radii", "gb_energy_forces", "redox_ph_mc_step", "eremd_exchange"):
        assert n in names


def test_every_declared_symbol_is_exported(lib):
    missing = [n for n in pkg.exported_names() if not hasattr(lib, n)]
    assert not missing, missing


def _header_struct_fields(name):
    src = open(pkg.HEADER).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    body = re.search(r"typedef struct \{([^{}]*)\}\s*" + name + ";", src).group(1)
    fields = []
    for decl in body.split(";"):
        decl = decl.strip()
        if not decl:
            continue
        parts = re.sub(r"^(const\s+)?[\w]+\s*\**\s*", "", decl)
        fields += [p.strip().lstrip("*") for p in parts.split(",")]
    return fields


@pytest.mark.parametrize("cname,pycls", [("gb_params", pkg.Params), ("gb_sites", pkg.Sites),
                                         ("gb_md_state", pkg.MDState), ("gb_md_host", pkg.MDHost)])
def test_struct_layouts_match_header(cname, pycls):
    assert _header_struct_fields(cname) == [f[0] for f in pycls._fields_]


def test_create_without_gpu_fails_cleanly(lib):
    """No CUDA device here: context creation must return an error code, not crash."""
    import torch
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    with pytest.raises(pkg.GBError):
        pkg.Context([0, 10])


@pytest.mark.parametrize("off,n_sites,msg", [
    ([1, 2, 3], 3, "site_off_host\\[0\\]"),
    ([0, 3, 2], 2, "non-decreasing"),
    ([0, 2, 4], 5, "must equal n_sites"),
    (None, 4, "site_off_host is NULL"),
])
def test_site_offsets_are_checked_on_the_host(lib, off, n_sites, msg):
    """gb_count_bound rejects a malformed replica -> site table before any
    CUDA call (the device pointers given here are never dereferenced)."""
    pkg.load()
    s = pkg.Sites()
    s.n_rep, s.n_sites = 2, n_sites
    arr = (ctypes.c_int32 * 3)(*off) if off is not None else None
    s.site_off_host = ctypes.cast(arr, ctypes.c_void_p) if arr is not None else None
    fake = 256                               # any non-NULL device address
    for k in ("site_off", "site_kind", "site_nstates", "site_state_off", "n_H", "n_e"):
        setattr(s, k, fake)
    rc = pkg.load().gb_count_bound(ctypes.byref(s), fake, 1, fake, None)
    assert rc == -1
    assert re.search(msg, pkg.load().gb_last_error(None).decode())
