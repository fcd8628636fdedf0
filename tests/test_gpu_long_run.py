"""The learned-collision forward pass over a long run (Eqs. S10-S12, with the
EDM forcing of Eq. S5): 1000 steps of a 256^2 periodic lattice, the
benchmark's recipe at that size (random divergence-free field with
E(k) ~ k^4 exp(-2 (k/8)^2) and rms 0.02, Kolmogorov forcing F0 = 1e-5 with
m = 4, tau = 0.6), for the benchmark's seeded Xavier weights and for the
trained weights: the BF16 tensor-core kernel and the FP32 CUDA-core kernel
against the FP64 oracle.

Checks:
* per step, on the run's own developed states: from the BF16 kernel's state
  at steps 500 and 999, one kernel step against one oracle step with the same
  bf16-rounded weights -- populations within ALPHA of the learned correction
  and velocity within TOL_U (the per-step tolerances of the one-step tests,
  with the same BGK guard);
* the whole run: each kernel's state after 1000 steps against the oracle's
  1000-step run with the weights the kernel computes with (bf16-rounded for
  BF16, FP32 for FP32).  Every figure is printed (the FP64 error of each
  result).
  - FP32 kernel: populations within 1e-5 of w_i.  Its only departures from
    the oracle are FP32 rounding (~6e-8 relative per operation) and tanhf
    (within 2 ulp), and the collision relaxes every non-conserved error
    (omega = 1/0.6), so per-step errors do not build up beyond a small
    multiple of one step's; 1e-5 is the bar of the FP32 BGK run.
  - BF16 kernel: its run must follow the learned model, i.e. stay at least 10x
    closer (velocity, relative L2) to the oracle's learned run than the
    oracle's BGK run is; a kernel that loses the network fails this.
  - both: total mass within 1e-6 (relative) of the start.
"""
import numpy as np
import pytest

import oracle
from paper_2403_18466_gb300 import inputs
from gpu_helpers import bf16_round, learned_pop_check, post_collision, rel_vel_err

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu
DEV = "cuda:0"
TOL_U = 2e-3
ALPHA = 5e-2
N, TAU, F0, MODE, STEPS = 256, 0.6, 1e-5, 4, 1000


@pytest.fixture(scope="module")
def lbm():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_2403_18466_gb300 import lbm as m
    m.load()
    return m


@pytest.fixture(scope="module")
def start():
    """Initial pre-collision state (the equilibrium of the random field), the
    oracle's stored form of it, and the oracle's 1000-step BGK run."""
    rho, ux, uy = inputs.random_velocity_field(N, N, seed=2, k0=8.0, urms=0.02)
    f0 = oracle.equilibrium_field(rho[None], ux[None], uy[None]).astype(np.float32)
    g0 = oracle.stream_push(f0.astype(np.float64))
    prm = oracle.params(TAU, force_amp=F0, force_mode=MODE)
    g_bgk = oracle.run(oracle.BGK, g0, STEPS, prm)
    return f0, g0, prm, g_bgk


def _dev(a):
    return torch.tensor(np.ascontiguousarray(a), dtype=torch.float32, device=DEV)


def _vel(g):
    _, ux, uy = oracle.moments(oracle.stream_pull(g))
    return ux, uy


def _rel_l2(u, v):
    (ux, uy), (vx, vy) = u, v
    return float(np.sqrt(((ux - vx) ** 2 + (uy - vy) ** 2).sum() / (vx ** 2 + vy ** 2).sum()))


def _weights(name):
    return inputs.xavier_mlp(3, out_scale=0.3) if name == "bench" else inputs.trained_mlp()


@pytest.mark.parametrize("weights", ["bench", "trained"])
def test_bf16_1000_steps_against_oracle(lbm, start, weights):
    f0, g0, prm, g_bgk = start
    theta = _weights(weights)
    thb = bf16_round(theta)
    _, _, wts = oracle.lattice()
    lat = lbm.Lattice(N, N, 1, tau=TAU, force_amp=F0, force_mode=MODE, device=DEV)
    w = lbm.weights_struct(_dev(theta))
    lat.set_state(_dev(f0))
    mass0 = float(f0.astype(np.float64).sum())
    done = 0
    for t in (500, 999):
        lat.step(t - done, "mlp_bf16", w)
        g = post_collision(lat)
        lat.step(1, "mlp_bf16", w)
        done = t + 1
        got = post_collision(lat)
        ref = oracle.step(oracle.MLP, g, prm, thb)
        ok, err, corr, tol = learned_pop_check(got, ref, oracle.step(oracle.BGK, g, prm), ALPHA)
        _, gx, gy = (a.double().cpu().numpy() for a in lat.moments())
        rx, ry = _vel(ref)
        eu = rel_vel_err(gx, gy, rx, ry)
        msg = (f"{weights} step {t}: pop err {err:.3e} (correction {corr:.3e}, err/corr "
               f"{err / corr:.3e}); velocity err {eu:.3e}")
        print(msg)
        assert corr > 10 * tol and ok, msg
        assert eu <= TOL_U, msg
    assert done == STEPS and lat.status() == lbm.LBM_OK
    g_ref = oracle.run(oracle.MLP, g0, STEPS, prm, thb)
    got = post_collision(lat)
    u_got, u_ref = lat.moments()[1:], _vel(g_ref)
    u_got = tuple(a.double().cpu().numpy() for a in u_got)
    d_kernel = _rel_l2(u_got, u_ref)
    d_bgk = _rel_l2(_vel(g_bgk), u_ref)
    d_pop = float(np.max(np.abs(got - g_ref) / wts[None, :, None, None]))
    mass = float(lat.get_state().double().sum())
    msg = (f"{weights} after {STEPS} steps: velocity rel L2 against the oracle's learned run "
           f"{d_kernel:.3e} (oracle BGK run {d_bgk:.3e}, ratio {d_kernel / d_bgk:.3e}), "
           f"populations {d_pop:.3e} of w_i, mass drift {mass / mass0 - 1:.2e}")
    print(msg)
    assert d_kernel <= 0.1 * d_bgk, msg
    assert abs(mass / mass0 - 1) <= 1e-6, msg


@pytest.mark.parametrize("weights", ["bench", "trained"])
def test_f32_1000_steps_against_oracle(lbm, start, weights):
    f0, g0, prm, g_bgk = start
    theta = _weights(weights)
    th32 = theta.astype(np.float32).astype(np.float64)
    _, _, wts = oracle.lattice()
    lat = lbm.Lattice(N, N, 1, tau=TAU, force_amp=F0, force_mode=MODE, device=DEV)
    lat.set_state(_dev(f0))
    lat.step(STEPS, "mlp_f32", lbm.weights_struct(_dev(theta)))
    assert lat.status() == lbm.LBM_OK
    g_ref = oracle.run(oracle.MLP, g0, STEPS, prm, th32)
    got = post_collision(lat)
    d_pop = float(np.max(np.abs(got - g_ref) / wts[None, :, None, None]))
    u_got = tuple(a.double().cpu().numpy() for a in lat.moments()[1:])
    d_u = _rel_l2(u_got, _vel(g_ref))
    d_bgk = _rel_l2(_vel(g_bgk), _vel(g_ref))
    mass0, mass = float(f0.astype(np.float64).sum()), float(lat.get_state().double().sum())
    msg = (f"{weights} FP32 after {STEPS} steps: populations {d_pop:.3e} of w_i, velocity rel "
           f"L2 {d_u:.3e} (oracle BGK run {d_bgk:.3e}), mass drift {mass / mass0 - 1:.2e}")
    print(msg)
    assert d_pop <= 1e-5, msg
    assert abs(mass / mass0 - 1) <= 1e-6, msg
