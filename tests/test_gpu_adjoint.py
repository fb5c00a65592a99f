"""Adjoint gradients of a detector response through torch.autograd against central finite
differences, on a log-normal sigma_t field with scattering ratio 0.99: FP64 sweeps, and the
gradient configuration's FP32 sweeps (each forward and adjoint SI-DSA sweep with its FP64 defect
correction; the psi and mu of the gradient contraction from FP32 sweeps of the converged
fluxes)."""
import numpy as np
import pytest

import workloads as W
from tests.helpers import oracle_disc

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


# the last case is the full 256 x 256, CL(64,8) gradient configuration with its 32 seeded directions
@pytest.mark.parametrize("prec", ["fp64", "fp32"])
@pytest.mark.parametrize("n,nt,nz,ndirs", [(24, 16, 4, 4), (64, 32, 4, 4), (256, 64, 8, 32)])
def test_autograd_gradient_matches_central_differences(n, nt, nz, ndirs, prec):
    from paper_2603_25233_gb300.api import Handle, detector_response
    spec = W.grf_adjoint_c5(n=n, n_theta=nt, n_omz=nz)
    d = oracle_disc(spec)
    det = torch.tensor(d.rect_functional(W.DETECTOR_C5), device="cuda")
    opts = dict(mode="fr", sweep_precision=prec, eps_si=1e-13, max_outer=2000, dsa_tol=1e-12)
    st0 = torch.tensor(spec.sig_t, dtype=torch.float64, requires_grad=True)
    ss0 = torch.tensor(spec.sig_s, dtype=torch.float64, requires_grad=True)
    q0 = torch.zeros(n * n, dtype=torch.float64, requires_grad=True)
    with Handle(spec) as h:
        R = detector_response(h, st0, ss0, q0, det, **opts)
        R.backward()
        gt, gs, gq = st0.grad.numpy(), ss0.grad.numpy(), q0.grad.numpy()
        dirs = W.random_unit_directions(ndirs, 2 * n * n, seed=20260105)
        hstep = 1e-4
        for v in dirs:
            vt, vs = v[:n * n], v[n * n:]
            vals = []
            for sgn in (1.0, -1.0):
                st = spec.sig_t * (1 + sgn * hstep * vt)
                ss = spec.sig_s * (1 + sgn * hstep * vs)
                with torch.no_grad():
                    vals.append(float(detector_response(h, torch.tensor(st), torch.tensor(ss),
                                                        torch.zeros(n * n, dtype=torch.float64), det, **opts)))
            fd = (vals[0] - vals[1]) / (2 * hstep)
            an = float(np.dot(gt, spec.sig_t * vt) + np.dot(gs, spec.sig_s * vs))
            assert abs(fd - an) <= 1e-4 * abs(an) + 1e-14, (fd, an)
        # source gradient: R is linear in q, so a single difference is exact
        e = np.zeros(n * n)
        e[0] = 1.0
        with torch.no_grad():
            Rq = float(detector_response(h, torch.tensor(spec.sig_t), torch.tensor(spec.sig_s),
                                         torch.tensor(e), det, **opts))
            R0 = float(detector_response(h, torch.tensor(spec.sig_t), torch.tensor(spec.sig_s),
                                         torch.zeros(n * n, dtype=torch.float64), det, **opts))
        assert abs((Rq - R0) - gq[0]) <= 1e-8 * abs(gq[0]) + 1e-15


def test_detector_functional_equals_the_source_moments_of_the_detector_square():
    """The detector functional d_k = int over [0.9,1]^2 of eta_k (the oracle's exact overlap
    integrals) is the source-moment vector of a problem whose only source is q = 1 on that square
    (how the benchmark forms d without the oracle)."""
    import dataclasses
    spec = W.grf_adjoint_c5(n=40, n_theta=8, n_omz=2)
    d = oracle_disc(spec)
    dspec = dataclasses.replace(spec, q_cell=None, q_rects=[tuple(W.DETECTOR_C5) + (1.0,)], q_gauss=[])
    from paper_2603_25233_gb300.api import Handle
    with Handle(dspec) as h:
        det = h.source().cpu().numpy()
    ref = d.rect_functional(W.DETECTOR_C5)
    assert np.abs(det - ref).max() <= 1e-14 * max(1.0, np.abs(ref).max())
