"""rd_cfl_dt (CFL time step of a caller-owned device state, Sec. 3.2) vs the oracle."""
import numpy as np
import pytest

import oracle
from paper_1705_02028_gb300 import inputs
from tests._gpu import mesh_device_arrays, require_gpu

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("N,state", [(64, "vortex"), (37, "khi"), (256, "sod"), (2, "sod")])
def test_cfl_dt_matches_oracle(N, state):
    torch = require_gpu()
    from paper_1705_02028_gb300 import binding
    mesh = inputs.periodic_grid(N, relabel_seed=4)
    W = {"vortex": inputs.vortex_state, "khi": inputs.khi_state, "sod": inputs.sod_like_state}[state](mesh)
    ref = oracle.time_step(mesh, W, cfl=0.8)
    for prec, dtype, tol in (("fp64", torch.float64, 1e-14), ("fp32", torch.float32, 2e-6)):
        a = mesh_device_arrays(mesh, torch, dtype)
        Wd = torch.tensor(W, dtype=dtype, device="cuda")
        dt = binding.cfl_dt(Wd, a["tri"], a["lmax"], a["V"], a["csr_ptr"], a["csr_ent"], precision=prec)
        assert dt == pytest.approx(ref, rel=tol), prec


def test_cfl_dt_reports_nonphysical_state():
    torch = require_gpu()
    from paper_1705_02028_gb300 import binding
    mesh = inputs.periodic_grid(8)
    W = inputs.uniform_state(mesh)
    W[3, 5] = -1.0
    a = mesh_device_arrays(mesh, torch, torch.float64)
    with pytest.raises(binding.RDError) as e:
        binding.cfl_dt(torch.tensor(W, device="cuda"), a["tri"], a["lmax"], a["V"], a["csr_ptr"], a["csr_ent"])
    assert e.value.status == binding.RD_ENONPHYSICAL
