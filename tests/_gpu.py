"""Helpers for the GPU tests: skip cleanly without a GPU, fail loudly without the library."""
import pytest


def require_gpu():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA GPU")
    from paper_1705_02028_gb300 import binding
    binding.load()  # raises if the CUDA library cannot be built or loaded
    return torch


def rel_max_err(a, b):
    """Per-component max|a-b| / max(max|b_k|, max|b_E|) (max norm, relative)."""
    import numpy as np
    scale = np.maximum(np.abs(b).max(axis=1), np.abs(b[3]).max())
    return float((np.abs(a - b).max(axis=1) / scale).max())


def mesh_device_arrays(mesh, torch, dtype):
    """Plain numpy construction (test-local) of the arrays rd_cfl_dt consumes:
    tri [3][nt], l_max [nt], V [nv] and the vertex -> corner CSR, on the GPU."""
    import numpy as np
    X = mesh.xy[mesh.tri][:, :, 0] + mesh.shift[:, :, 0] * mesh.Lx
    Y = mesh.xy[mesh.tri][:, :, 1] + mesh.shift[:, :, 1] * mesh.Ly
    edges = [np.hypot(X[:, (c + 2) % 3] - X[:, (c + 1) % 3], Y[:, (c + 2) % 3] - Y[:, (c + 1) % 3]) for c in range(3)]
    lmax = np.max(np.stack(edges), axis=0)
    area = 0.5 * ((X[:, 1] - X[:, 0]) * (Y[:, 2] - Y[:, 0]) - (X[:, 2] - X[:, 0]) * (Y[:, 1] - Y[:, 0]))
    V = np.zeros(mesh.nv)
    np.add.at(V, mesh.tri.ravel(), np.repeat(area / 3.0, 3))
    corner = np.arange(3 * mesh.nt, dtype=np.int64)          # 3 t + c
    order = np.argsort(mesh.tri.ravel(), kind="stable")
    ptr = np.zeros(mesh.nv + 1, dtype=np.int64)
    np.add.at(ptr, mesh.tri.ravel() + 1, 1)
    ptr = np.cumsum(ptr)
    dev = "cuda"
    return dict(tri=torch.tensor(np.ascontiguousarray(mesh.tri.T), dtype=torch.int32, device=dev),
                lmax=torch.tensor(lmax, dtype=dtype, device=dev), V=torch.tensor(V, dtype=dtype, device=dev),
                csr_ptr=torch.tensor(ptr, dtype=torch.int32, device=dev),
                csr_ent=torch.tensor(corner[order], dtype=torch.int32, device=dev))
