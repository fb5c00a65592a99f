"""Launch configurations of the sweep and their autotuner (rte_sweep_tune, rte_sweep_set_config,
rte_sweep_get_config).  The sweep of Sec. 2.2 is the same per-cell computation in every
configuration: psi must be bit-identical across the band kernel's configurations (bands in
flight, prefetch depth, staged or direct stores), and every configuration, band or warp kernel,
must match the oracle's direct solve of each upwind system.  The tuner must pick a valid
configuration, an uncaptured sweep of a new kind must tune itself, and invalid configurations
must be refused."""
import numpy as np
import pytest

import workloads as W
from tests.helpers import gpu_handle, oracle_disc, rel_l2

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

FP64, FP32 = 0, 1
TOL = {FP64: 1e-12, FP32: 2e-5}


def _spec(nx, ny, seed=0, nt=8, nz=2):
    return W.random_small(nx, ny, n_theta=nt, n_omz=nz, seed=seed, inflow=(0.3, 0.1, 0.2, 0.4),
                          box=(0.0, 1.3, -0.2, 0.9))


def _expected_valid(cfg, nx, ny, esz):
    if cfg["kernel"] == "warp":
        return 2 * nx * esz * cfg["angles_per_block"] <= 200 * 1024
    nb = (ny + 31) // 32
    W_, D = cfg["warps"], cfg["depth"]
    if not (nx >= 32 and ny > 32) or W_ < 1 or W_ > 16 or W_ > nb or cfg["angles_per_block"] not in (1, 2, 4):
        return False
    if W_ < nb and nx < 32 * W_ + 4:
        return False
    return True          # shared memory checked by the library (the test meshes fit)


def _all_configs(nx, ny):
    out = [dict(kernel="warp", warps=0, depth=0, staged=0, angles_per_block=a) for a in (1, 2, 4)]
    nb = (ny + 31) // 32
    for W_ in sorted({1, 2, 3, 4, 7, 8, 16, nb, nb + 1}):
        for D in (2, 4, 8):
            for sg in (0, 1):
                out.append(dict(kernel="band", warps=W_, depth=D, staged=sg, angles_per_block=1))
    # persistent band grids: 4 blocks of 2 ordinates, 2 blocks of 4
    out += [dict(kernel="band", warps=min(nb, 16) if nb <= 16 else 1, depth=4, staged=sg, angles_per_block=a)
            for a in (2, 4) for sg in (0, 1)]
    return out


def _sweep(h, angles, S, prec, nd):
    psi = torch.empty(len(angles) * nd, dtype=torch.float64 if prec == FP64 else torch.float32, device="cuda")
    h.sweep(angles, S, prec, src_per_angle=True, psi_out=psi)
    torch.cuda.synchronize()
    return psi


# a single band, several bands (ragged), bands > 32 W + 4 columns wide, more than 16 bands
# (cyclic band ownership only), and a mesh below one band (warp kernel only)
@pytest.mark.parametrize("prec", [FP64, FP32])
@pytest.mark.parametrize("shape", [(40, 33), (150, 200), (36, 100), (20, 20), (300, 600)])
def test_every_sweep_configuration_gives_the_same_psi(shape, prec):
    from paper_2603_25233_gb300._lib import RteError
    nx, ny = shape
    spec = _spec(nx, ny, seed=3)
    esz = 8 if prec == FP64 else 4
    angles = np.array([0, 3, 5, 6, 9, 12, 14, 15])
    with gpu_handle(spec) as h:
        nd = h.n_dof
        rng = np.random.default_rng(4)
        S64 = rng.standard_normal(len(angles) * nd)
        S = torch.tensor(S64, device="cuda", dtype=torch.float64 if prec == FP64 else torch.float32)
        n = len(angles)
        ref_band = None
        ref = None
        if nx * ny <= 40000:
            from oracle.transport import DirectSweeper
            d = oracle_disc(spec)
            sw = DirectSweeper(d)
            ref = [sw.sweep(int(j), S64[a * nd:(a + 1) * nd]) for a, j in enumerate(angles)]
        for cfg in _all_configs(nx, ny):
            ok = _expected_valid(cfg, nx, ny, esz)
            if not ok:
                with pytest.raises(RteError):
                    h.sweep_set_config(prec, n, True, cfg)
                continue
            h.sweep_set_config(prec, n, True, cfg)
            assert {k: v for k, v in h.sweep_get_config(prec, n, True).items() if k != "ms"} == cfg
            psi = _sweep(h, angles, S, prec, nd)
            if cfg["kernel"] == "band":
                if ref_band is None:
                    ref_band = psi.clone()
                else:
                    assert torch.equal(psi, ref_band), cfg
            if ref is not None:
                P = psi.double().cpu().numpy().reshape(n, nd)
                for a in range(n):
                    assert rel_l2(P[a], ref[a]) < TOL[prec], (cfg, a)
        # malformed configurations
        for bad in (dict(kernel="band", warps=1, depth=3, staged=0, angles_per_block=1),
                    dict(kernel="band", warps=1, depth=4, staged=2, angles_per_block=1),
                    dict(kernel="warp", warps=0, depth=0, staged=0, angles_per_block=3),
                    dict(kernel="band", warps=1, depth=4, staged=0, angles_per_block=3),
                    dict(kernel=7, warps=1, depth=4, staged=0, angles_per_block=1)):
            with pytest.raises(RteError):
                h.sweep_set_config(prec, n, True, bad)


@pytest.mark.parametrize("prec", [FP64, FP32])
def test_tuner_picks_a_valid_configuration_and_sweeps_tune_themselves(prec):
    nx, ny = 150, 200
    spec = _spec(nx, ny, seed=5)
    angles = np.arange(8)
    with gpu_handle(spec) as h:
        nd = h.n_dof
        n = len(angles)
        cfg = h.sweep_tune(prec, n, True)
        assert cfg["ms"] > 0 and _expected_valid(cfg, nx, ny, 8 if prec == FP64 else 4)
        assert h.sweep_get_config(prec, n, True) == cfg
        # forget it: the next uncaptured sweep of that kind tunes itself and caches the result
        h.sweep_set_config(prec, n, True, None)
        assert h.sweep_get_config(prec, n, True)["ms"] == 0
        S = torch.ones(n * nd, device="cuda", dtype=torch.float64 if prec == FP64 else torch.float32)
        psi = _sweep(h, angles, S, prec, nd)
        tuned = h.sweep_get_config(prec, n, True)
        assert tuned["ms"] > 0
        # the tuned sweep equals the default configuration's, bit for bit (band kernel)
        default = dict(kernel="band", warps=7, depth=4, staged=0, angles_per_block=1)
        h.sweep_set_config(prec, n, True, default)
        assert torch.equal(_sweep(h, angles, S, prec, nd), psi) or tuned["kernel"] == "warp"


def test_lowrank_solve_tunes_its_p_ordinate_sweeps_before_capturing():
    """A low-rank solve (its inner-loop sweeps run inside graph captures) tunes the p-ordinate
    launches first; the solve equals the one with the default configuration forced."""
    spec = _spec(64, 48, seed=6, nt=16, nz=2)
    opts = dict(mode="lr", sweep_precision="fp32", sweep_refine=1, eps_si=1e-8, eps_res=1e-9, eps_diff=1e-9,
                p=4, q=8, seed=2)
    with gpu_handle(spec) as h:
        assert h.sweep_get_config(FP32, 4, True)["ms"] == 0
        phi1, st1 = h.si_dsa_solve(**opts)
        assert h.sweep_get_config(FP32, 4, True)["ms"] > 0
        h.sweep_set_config(FP32, 4, True, dict(kernel="band", warps=2, depth=4, staged=0, angles_per_block=1))
        phi2, st2 = h.si_dsa_solve(**opts)
    assert st1["total_inner"] == st2["total_inner"] and st1["max_rank"] == st2["max_rank"]
    assert torch.equal(phi1, phi2)
