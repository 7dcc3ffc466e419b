"""The adjoint's hand-written reverse of the per-triangle code (the functions the
reverse kernels call), compiled for the host and checked without a GPU by the
dot-product test: for seeded random triangles, output adjoints and input
directions, <out_bar, J dx> from central differences of the forward
per-triangle code equals <J^T out_bar, dx> from the reverse code.  Stage 1
(Z -> shares and stage-1 record) and stage 2 (Z*, W^n, W*, record -> shares)
for the N, B and LDA schemes; triangles whose branch mask changes within the
difference step are skipped (the map has a kink there)."""
import os
import shutil
import subprocess

import pytest

from paper_1705_02028_gb300 import build

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)


def test_reverse_code_dot_product():
    nvcc = shutil.which("nvcc") or ("/usr/local/cuda/bin/nvcc" if os.path.exists("/usr/local/cuda/bin/nvcc") else None)
    if not nvcc:
        pytest.skip("nvcc not available")
    exe = os.path.join(os.environ.get("TMPDIR", "/tmp"), "adjoint_host_check_%d" % os.getpid())
    subprocess.run([nvcc, "-std=c++17", "-O2", "-gencode", "arch=compute_103a,code=sm_103a", "-I", build.CSRC,
                    "-I", os.path.join(ROOT, "include"), os.path.join(HERE, "adjoint_host_check.cu"), "-o", exe],
                   check=True)
    try:
        out = subprocess.run([exe, "800"], capture_output=True, text=True, check=True).stdout
    finally:
        os.remove(exe)
    print(out)
    rows = [ln.split() for ln in out.strip().splitlines()]
    assert len(rows) == 5  # N1 stage 1; B2 and LDA2 stages 1 and 2
    for scheme, stage, _, checked, _, skipped, _, err in rows:
        assert int(checked) >= 100, (scheme, stage, checked, skipped)
        assert float(err) < 1e-7, (scheme, stage, err)
