"""Shared helpers of the GPU parity tests (oracle parameters rounded to the
FP32 values the library receives, tolerances, device set-up)."""
import numpy as np

import oracle

KT = oracle.KB * 300.0

# Tolerances (spec values): energy relative 1e-6, forces 1e-3
# kcal/mol/A max-abs, state-change energy 1e-3 kcal/mol.
E_REL = 1e-6
F_ABS = 1e-3
DG_ABS = 1e-3
# Born radii are FP32 results of FP32 pair sums: a few ulp of R.
R_REL = 2e-6
# dE/dq: FP32 pair terms of magnitude up to ~k_e/r summed in fixed point
PHI_ABS = 2e-3


def f32(v):
    return float(np.float32(v))


def oracle_params(**kw):
    """Oracle parameters equal to the float32 values the CUDA library stores."""
    d = dict(alpha=f32(1.0), beta=f32(0.8), gamma=f32(4.85), offset=f32(0.09), eps_in=1.0,
             eps_out=78.5)
    d.update(kw)
    return oracle.default_params(**d)


def device():
    import torch
    if not torch.cuda.is_available():
        import pytest
        pytest.skip("no CUDA device")
    return torch.device("cuda:0")


def to_dev(batch, dev):
    import torch
    return (torch.as_tensor(batch.xyzq(), device=dev), torch.as_tensor(batch.rad_screen(), device=dev))


def energy_rel_err(E_gpu, E_ref):
    """Per replica |dE| / |E| of E_GB + E_Coul (E_gpu: [M,3] GB, Coul, rep)."""
    tot_g = E_gpu[:, 0] + E_gpu[:, 1]
    tot_r = E_ref[:, 0] + E_ref[:, 1]
    return np.abs(tot_g - tot_r) / np.maximum(np.abs(tot_r), 1e-30)
