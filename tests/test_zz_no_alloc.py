"""The allocation-free entry point gb_energy_forces_static, called through the
C ABI, against the context-based gb_energy_forces on the same molecule.

It exists for callers that cannot call cudaMalloc (device memory owned by an
arena allocator, plugins barred from allocating after start-up, real-time
loops); its workspace is a static device array shared by every call, so two
calls in a row must both reproduce the context path -- the second one starting
from whatever the first left in the array.  Kept in a file of its own that
collects last."""
import ctypes as C

import numpy as np
import pytest

import oracle
import synth
from gpu_common import E_REL, F_ABS, PHI_ABS, R_REL, device, energy_rel_err, oracle_params

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def lib():
    import __graft_entry__
    __graft_entry__.build()
    import paper_1803_09652_gb300 as pkg
    lib = pkg.load()
    f = lib.gb_energy_forces_static
    P = C.c_void_p
    f.argtypes = [C.c_int32, C.POINTER(pkg.Params), P, P, P, P, P, P, P, P]
    f.restype = C.c_int
    return lib


def _outputs(n, dev):
    import torch
    return dict(R=torch.full((n,), float("nan"), dtype=torch.float32, device=dev),
               F=torch.full((n, 3), float("nan"), dtype=torch.float32, device=dev),
               F_fixed=torch.zeros((3, n), dtype=torch.int64, device=dev),
               E=torch.full((1, 3), float("nan"), dtype=torch.float64, device=dev),
               dEdq=torch.full((n,), float("nan"), dtype=torch.float64, device=dev))


def _static_call(lib, pkg, params, n, xyzq, rad, out=None):
    import torch
    out = out or _outputs(n, xyzq.device)
    s = torch.cuda.current_stream().cuda_stream
    rc = lib.gb_energy_forces_static(n, C.byref(params), xyzq.data_ptr(), rad.data_ptr(),
                                     out["R"].data_ptr(), out["F_fixed"].data_ptr(),
                                     out["F"].data_ptr(), out["E"].data_ptr(), out["dEdq"].data_ptr(), s)
    assert rc == 0
    torch.cuda.synchronize()
    return {k: v.cpu().numpy() for k, v in out.items()}


def _check(a, ref):
    e_a, e_r = a["E"][0, 0] + a["E"][0, 1], ref["E"][0, 0] + ref["E"][0, 1]
    assert abs(e_a - e_r) <= E_REL * abs(e_r)
    assert np.abs(a["F"] - ref["F"]).max() <= F_ABS
    assert np.max(np.abs(a["R"] - ref["R"]) / ref["R"]) <= R_REL
    assert np.abs(a["dEdq"] - ref["dEdq"]).max() <= PHI_ABS


def test_static_entry_matches_context_entry_twice(lib):
    import torch
    import paper_1803_09652_gb300 as pkg
    dev = device()
    params = pkg.default_params(rep_k=100.0, rep_sigma=2.5)
    mols = [synth.random_batch([700], seed=31), synth.random_batch([1500], seed=32)]
    refs = []
    for b in mols:
        xyzq = torch.as_tensor(b.xyzq(), device=dev)
        rad = torch.as_tensor(b.rad_screen(), device=dev)
        ctx = pkg.Context(b.atom_off, params)
        o = ctx.energy_forces(xyzq, rad)
        torch.cuda.synchronize()
        refs.append(({k: v.cpu().numpy() for k, v in o.items()}, xyzq, rad, b.n_atoms))
        ctx.close()
    # two calls in a row on each molecule, the second molecule after the first
    for ref, xyzq, rad, n in refs:
        for _ in range(2):
            a = _static_call(lib, pkg, params, n, xyzq, rad)
            _check(a, ref)


def test_static_entry_rejects_sizes_beyond_the_limit(lib):
    import torch
    import paper_1803_09652_gb300 as pkg
    dev = device()
    params = pkg.default_params()
    n = 8193
    xyzq = torch.zeros((n, 4), dtype=torch.float32, device=dev)
    rad = torch.ones((n, 2), dtype=torch.float32, device=dev)
    R = torch.zeros(n, dtype=torch.float32, device=dev)
    s = torch.cuda.current_stream().cuda_stream
    rc = lib.gb_energy_forces_static(n, C.byref(params), xyzq.data_ptr(), rad.data_ptr(), R.data_ptr(),
                                     None, None, None, None, s)
    assert rc == pkg.GBError(-1, "").code == -1
    rc = lib.gb_energy_forces_static(0, C.byref(params), xyzq.data_ptr(), rad.data_ptr(), R.data_ptr(),
                                     None, None, None, None, s)
    assert rc == -1


@pytest.mark.parametrize("n", [8192, 8191, 8129])
def test_static_entry_at_its_size_limit(lib, n):
    """At the limit (n = 8192: the largest task list and every sub-buffer of
    the array full), one atom short of it, and at 8129 atoms (255 tiles, the
    last holding one atom): two calls in a row against a context, and
    against the FP64 oracle element by element."""
    import torch
    import paper_1803_09652_gb300 as pkg
    dev = device()
    params = pkg.default_params()
    b = synth.Batch([synth.make_replica(n, 60 + n % 7, [])], pH=np.array([7.0]), E=np.array([synth.E0_REF_V]))
    xyzq = torch.as_tensor(b.xyzq(), device=dev)
    rad = torch.as_tensor(b.rad_screen(), device=dev)
    ctx = pkg.Context(b.atom_off, params)
    ref = {k: v.cpu().numpy() for k, v in ctx.energy_forces(xyzq, rad).items()}
    ctx.close()
    for _ in range(2):
        a = _static_call(lib, pkg, params, n, xyzq, rad)
        _check(a, ref)
    x, q, rho, scr, off = oracle.batch_arrays(b)
    o = oracle.energy_forces(x, q, rho, scr, oracle_params())
    assert energy_rel_err(a["E"], o["E"][None, :]).max() <= E_REL
    assert np.abs(a["F"] - o["F"]).max() <= F_ABS
    assert np.max(np.abs(a["R"] - o["R"]) / o["R"]) <= R_REL
    assert np.abs(a["dEdq"] - o["phi"]).max() <= PHI_ABS


def test_static_entry_allocates_no_device_memory(lib):
    """Free device memory is the same before and after a warmed-up call (the
    outputs are allocated beforehand, as such a caller would hold them)."""
    import torch
    import paper_1803_09652_gb300 as pkg
    dev = device()
    params = pkg.default_params()
    b = synth.random_batch([4000], seed=33, sites=False)
    xyzq = torch.as_tensor(b.xyzq(), device=dev)
    rad = torch.as_tensor(b.rad_screen(), device=dev)
    out = _outputs(b.n_atoms, dev)
    _static_call(lib, pkg, params, b.n_atoms, xyzq, rad, out)
    torch.cuda.synchronize()
    free0 = torch.cuda.mem_get_info()[0]
    _static_call(lib, pkg, params, b.n_atoms, xyzq, rad, out)
    torch.cuda.synchronize()
    assert torch.cuda.mem_get_info()[0] == free0
