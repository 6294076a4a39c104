"""Helpers shared by the GPU parity tests (inputs, oracle calls, tolerances)."""
import numpy as np
import torch

import oracle
from paper_2408_16847_gb300 import tpcf

# Parity bar, per multipole: for every m, max_{k1,k2} |zeta_gpu - zeta_oracle| must stay
# below TOL * max_{k1,k2} |zeta_oracle| of that same m (each multipole against its own
# largest entry), and likewise for the raw sums S and the gradient.
TOL = 1e-5


def to_dev(a, dtype=torch.float32):
    return torch.from_numpy(np.ascontiguousarray(a)).to("cuda:0", dtype)


def rel_err_per_m(zg, zo):
    """Per-m relative error max_k |dz| / max_k |z_oracle| (m where the oracle is all zero: abs)."""
    out = []
    for m in range(zo.shape[0]):
        s = np.abs(zo[m]).max()
        d = np.abs(zg[m] - zo[m]).max()
        out.append(d / s if s > 0 else d)
    return np.array(out)


def gpu_zeta(plan, d32, w32, pivots=None):
    zeta, norm = plan.forward(to_dev(d32), to_dev(w32), pivots)
    torch.cuda.synchronize()
    plan.sync()
    return tpcf.as_complex(zeta).cpu().numpy(), norm.cpu().numpy()
