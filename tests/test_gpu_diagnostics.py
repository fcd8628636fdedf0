"""GPU parity of the flow diagnostics (structure functions, energy spectrum)
against the oracle, and the Smagorinsky-LES spectrum check of the 1024^2
configuration at 128^2 (same recipe, GPU run vs oracle run).

Tolerances: the GPU works from FP32 populations, the oracle in FP64 from the
same FP32 populations; sums are reordered.  Even structure functions and the
spectrum: 1e-4 relative; odd structure functions (small by cancellation): 1e-4
of the mean |du|^p.  After 200 Smagorinsky steps the spectra of the two runs:
1e-3 relative on every shell holding more than 1e-6 of the peak energy.
"""
import numpy as np
import pytest

import oracle
from paper_2403_18466_gb300 import inputs
from gpu_helpers import population_field

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu
DEV = "cuda:0"


@pytest.fixture(scope="module")
def lbm():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_2403_18466_gb300 import lbm as m
    m.load()
    return m


def _dev(a):
    return torch.tensor(np.ascontiguousarray(a), dtype=torch.float32, device=DEV)


@pytest.mark.parametrize("nx,ny,B,rmax", [(64, 48, 2, 20), (37, 29, 1, 30), (300, 8, 1, 5)])
def test_structure_functions_parity(lbm, nx, ny, B, rmax):
    f = population_field(B, ny, nx, seed=91, urms=0.04)
    lat = lbm.Lattice(nx, ny, B, device=DEV)
    lat.set_state(_dev(f))
    S = lat.structure_functions(rmax).cpu().numpy()
    _, vx, vy = oracle.moments(lat.get_state().double().cpu().numpy())
    R = oracle.structure_functions(vx, vy, rmax)
    for p in range(1, 7):
        if p % 2 == 0:
            assert np.allclose(S[p - 1], R[p - 1], rtol=1e-4, atol=0), p
        else:
            for r in range(1, rmax + 1):
                dx = np.roll(vx, -r, axis=2) - vx
                dy = np.roll(vy, -r, axis=1) - vy
                scale = 0.5 * np.mean(np.abs(dx) ** p + np.abs(dy) ** p)
                assert abs(S[p - 1, r - 1] - R[p - 1, r - 1]) <= 1e-4 * scale, (p, r)


@pytest.mark.parametrize("nx,ny,B", [(64, 64, 1), (96, 40, 2), (33, 35, 1)])
def test_energy_spectrum_parity(lbm, nx, ny, B):
    f = population_field(B, ny, nx, seed=92, urms=0.03, k0=5.0)
    lat = lbm.Lattice(nx, ny, B, device=DEV)
    lat.set_state(_dev(f))
    kmax = int(np.ceil(np.hypot(nx, ny) / 2)) + 1
    E = lat.energy_spectrum(kmax).cpu().numpy()
    _, vx, vy = oracle.moments(lat.get_state().double().cpu().numpy())
    R = oracle.energy_spectrum(vx, vy, kmax)
    big = R > 1e-6 * R.max()
    assert np.allclose(E[big], R[big], rtol=1e-4)
    assert np.all(np.abs(E[~big]) <= 1e-4 * R.max())
    assert np.isclose(E.sum(), 0.5 * np.mean(vx ** 2 + vy ** 2), rtol=1e-4)


def test_smagorinsky_les_spectrum_at_128_matches_oracle(lbm):
    """The 1024^2 Smagorinsky configuration (tau0 = 0.51, C_s = 0.1, Kolmogorov
    F0 = 1e-5 at m = 4, random field rms 0.02, seed 1) checked at 128^2: GPU run
    vs oracle run, 200 steps, energy spectra compared."""
    n, steps, tau, cs, F0, m = 128, 200, 0.51, 0.1, 1e-5, 4
    rho, ux, uy = inputs.random_velocity_field(n, n, seed=1, k0=8.0, urms=0.02)
    lat = lbm.Lattice(n, n, 1, tau=tau, smag_cs=cs, force_amp=F0, force_mode=m, device=DEV)
    lat.init_equilibrium(_dev(rho[None]), _dev(ux[None]), _dev(uy[None]))
    g = oracle.stream_push(lat.get_state().double().cpu().numpy())
    lat.step(steps, "smag")
    g = oracle.run(oracle.SMAG, g, steps, oracle.params(tau, smag_cs=cs, force_amp=F0,
                                                        force_mode=m))
    kmax = 91
    E = lat.energy_spectrum(kmax).cpu().numpy()
    _, vx, vy = oracle.moments(oracle.stream_pull(g))
    R = oracle.energy_spectrum(vx, vy, kmax)
    big = R > 1e-6 * R.max()
    assert np.allclose(E[big], R[big], rtol=1e-3)
    assert lat.status() == lbm.LBM_OK


def test_les_run_records_statistics(lbm):
    """The long-run driver: spectra and structure functions every `every`
    steps, finite, S^2 positive and rising at small r, and the ESS slope of S^3
    against itself equal to one."""
    from paper_2403_18466_gb300 import les
    res = les.run(n=64, kind="smag", steps=300, every=100, rmax=12, kmax=46)
    assert res["steps"] == [100, 200, 300]
    assert res["E"].shape == (3, 47) and res["S"].shape == (3, 6, 12)
    assert np.all(np.isfinite(res["E"])) and np.all(np.isfinite(res["S"]))
    assert res["status"] == lbm.lbm_strerror(lbm.LBM_OK)
    # S^2 > 0 and grows with r at small separations in a smooth field
    assert np.all(res["S"][:, 1, :] > 0) and np.all(np.diff(res["S"][-1, 1, :4]) > 0)
    xi = les.ess_exponents(res["S"].mean(0))
    assert abs(xi[2] - 1.0) < 1e-12 and np.all(np.isfinite(xi))


def test_long_comparison_reports_the_unstable_step(lbm):
    """The long-run comparison stops a run at the first status check (every
    check_every steps) that finds |u| >= 0.4 or a non-finite value and reports
    that step; statistics are kept only for the records before it.  A learned
    collision with an oversized output layer blows up; Smagorinsky at tau 0.6
    does not."""
    from paper_2403_18466_gb300 import inputs, les
    theta = torch.tensor(inputs.xavier_mlp(3, out_scale=3.0), dtype=torch.float32, device=DEV)
    rec = les.long_comparison(theta, n=64, steps=600, every=200, tau=0.6, rmax=8,
                              device=DEV, check_every=50)
    ml, sm = rec["mlp_bf16"], rec["smag"]
    assert ml["unstable_at"] is not None and ml["unstable_at"] % 50 == 0
    assert ml["unstable_at"] <= 600
    assert all(s < ml["unstable_at"] for s in ml["steps"])
    assert len(ml["steps"]) == (ml["unstable_at"] - 1) // 200
    assert sm["unstable_at"] is None and sm["steps"] == [200, 400, 600]
    assert np.all(np.isfinite(sm["energy"])) and sm["ess"] is not None
