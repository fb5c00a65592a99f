"""The tensor-core projection X^T Psi (tcgen05, split-TF32 operands, FP32 accumulation in tensor
memory) against FP64 sums of the same FP32 entries: every sum within a few 1e-7 of the sum of
absolute products (plain TF32 would be ~1e-3).  Ragged row counts (not a multiple of the 32-row
tiles or of the 1024-row blocks), several 128-column tiles, 1 to 8 vectors."""
import numpy as np
import pytest

import workloads as W
from tests.helpers import gpu_handle

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("shape,r,nv", [((37, 29), 1, 1), ((37, 29), 100, 5), ((64, 64), 128, 8),
                                        ((64, 64), 130, 8), ((40, 33), 300, 3), ((3, 1), 7, 8)])
def test_basis_project_matches_fp64_sums(shape, r, nv):
    spec = W.random_small(*shape, seed=1)
    with gpu_handle(spec) as h:
        N = h.n_dof
        g = torch.Generator(device="cuda").manual_seed(r * 31 + nv)
        X = torch.randn(r, N, dtype=torch.float32, device="cuda", generator=g)
        X[::3] *= 1e-3                                           # mixed magnitudes across columns
        P = torch.randn(nv, N, dtype=torch.float32, device="cuda", generator=g)
        out = h.basis_project(X, P).cpu().numpy()
        out2 = h.basis_project(X, P).cpu().numpy()               # same launch again: same result
    Xd = X.double().cpu().numpy()
    Pd = P.double().cpu().numpy()
    ref = Pd @ Xd.T                                              # [nv, r]
    scale = np.abs(Pd) @ np.abs(Xd).T
    assert np.all(np.abs(out - ref) <= 2e-6 * scale + 1e-30)
    assert np.array_equal(out, out2)
    # the split scheme is far more accurate than plain TF32 (~2^-11 per product)
    assert np.max(np.abs(out - ref) / scale) < 1e-5


def test_basis_project_rejects_bad_arguments():
    from paper_2603_25233_gb300 import _lib as L
    spec = W.random_small(8, 8, seed=2)
    with gpu_handle(spec) as h:
        X = torch.zeros(4, h.n_dof, dtype=torch.float32, device="cuda")
        P = torch.zeros(9, h.n_dof, dtype=torch.float32, device="cuda")
        with pytest.raises(L.RteError):
            h.basis_project(X, P)                                 # more than 8 vectors
