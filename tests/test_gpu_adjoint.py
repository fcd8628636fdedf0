"""GPU parity of the hand-written adjoint (unrolled training, SI section 2)
against the oracle's reverse mode, which is itself pinned by central finite
differences (tests/test_oracle_adjoint.py).

Tolerance: 1e-4 relative (infinity norm) on dL/dtheta and on dL/df0, from
FP32 accumulation over the unroll; the loss to 1e-5.
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


def _np(t):
    return t.double().cpu().numpy()


@pytest.mark.parametrize("nx,ny,B,steps,ck", [(24, 16, 2, 5, 2), (160, 12, 1, 4, 4), (32, 32, 1, 3, 1)])
def test_backward_matches_oracle(lbm, nx, ny, B, steps, ck):
    tau, F0, m = 0.6, 1e-4, 1
    theta = inputs.xavier_mlp(7, bias_scale=0.3, gain=3.0, out_scale=0.01)
    th32 = theta.astype(np.float32).astype(np.float64)
    f0 = population_field(B, ny, nx, seed=61, neq=0.05)
    utx = inputs.noise((B, ny, nx), 62, 0.03).astype(np.float32)
    uty = inputs.noise((B, ny, nx), 63, 0.03).astype(np.float32)

    lat = lbm.Lattice(nx, ny, B, tau=tau, force_amp=F0, force_mode=m, device=DEV)
    th = _dev(theta)
    w = lbm.weights_struct(th)
    lat.set_state(_dev(f0))
    ws = torch.empty(lat.record_bytes(steps, ck) // 4, dtype=torch.float32, device=DEV)
    lat.forward_record(steps, ck, w, ws)
    loss, dL_df = lat.velocity_loss(_dev(utx), _dev(uty))
    dW = torch.empty(lbm.LBM_MLP_NPARAMS, dtype=torch.float32, device=DEV)
    dF0 = torch.empty_like(dL_df)
    lat.backward(dL_df, w, ws, dW, dF0)
    assert lat.status() == lbm.LBM_OK

    prm = oracle.params(tau, force_amp=F0, force_mode=m)
    g0 = oracle.stream_push(f0.astype(np.float64))
    L, dth, dg0 = oracle.unroll_grad(g0, steps, prm, th32, utx.astype(np.float64),
                                     uty.astype(np.float64))
    assert abs(float(loss.item()) / L - 1) <= 1e-5
    dWg = _np(dW)
    assert np.abs(dWg - dth).max() <= 1e-4 * np.abs(dth).max()
    df0 = oracle.stream_pull(dg0)
    assert np.abs(_np(dF0) - df0).max() <= 1e-4 * np.abs(df0).max()
    # the forward that was recorded is the plain learned-collision run
    lat2 = lbm.Lattice(nx, ny, B, tau=tau, force_amp=F0, force_mode=m, device=DEV)
    lat2.set_state(_dev(f0))
    lat2.step(steps, "mlp_f32", w)
    assert torch.equal(lat2.get_state(), lat.get_state())
    # deterministic: a second backward gives the same bits
    dW2 = torch.empty_like(dW)
    lat.backward(dL_df, w, ws, dW2, None)
    assert torch.equal(dW, dW2)


@pytest.mark.parametrize("nx,ny,B,steps,ck", [(24, 16, 2, 5, 2), (300, 20, 1, 4, 4), (128, 128, 1, 3, 1),
                                              (1024, 128, 1, 2, 1)])
@pytest.mark.parametrize("record", ["f32", "bf16"])
def test_tensor_core_backward_matches_oracle(lbm, nx, ny, B, steps, ck, record):
    """Tensor-core adjoint (tcgen05 GEMMs, bf16 operands) against the oracle's
    reverse mode with the same bf16-rounded weights.

    Tolerance 5e-2 relative L2 on dtheta and on dL/df0 (2.5x that per
    parameter block; cosine >= 0.995).  Derivation: for the velocity loss the
    adjoint entering each step lies mostly in the conserved span {1, c_x, c_y},
    so dL/do after the projection is small and the weight gradients are sums
    over nodes with strong cancellation; a numpy emulation of this very case
    (exact arithmetic except bf16 rounding at the kernel's rounding points:
    x, h, 1 - h^2, dL/do, dL/da) is 2.3e-2 off the exact gradient for one
    step (b1 3.7e-2, W3 2.4e-2), mostly from rounding h and dL/do, and the
    error compounds mildly over steps.  record "f32" isolates the adjoint
    (states as the oracle's); record "bf16" is the whole tensor-core pair."""
    from gpu_helpers import bf16_round
    tau, F0, m = 0.6, 1e-4, 1
    theta = inputs.xavier_mlp(7, bias_scale=0.3, gain=3.0, out_scale=0.01)
    thb = bf16_round(theta)
    f0 = population_field(B, ny, nx, seed=81, neq=0.05)
    utx = inputs.noise((B, ny, nx), 82, 0.03).astype(np.float32)
    uty = inputs.noise((B, ny, nx), 83, 0.03).astype(np.float32)
    lat = lbm.Lattice(nx, ny, B, tau=tau, force_amp=F0, force_mode=m, device=DEV)
    w = lbm.weights_struct(_dev(thb))
    lat.set_state(_dev(f0))
    ws = torch.empty(lat.record_bytes(steps, ck) // 4, dtype=torch.float32, device=DEV)
    lat.forward_record(steps, ck, w, ws, record)
    loss, dL_df = lat.velocity_loss(_dev(utx), _dev(uty))
    dW = torch.empty(lbm.LBM_MLP_NPARAMS, dtype=torch.float32, device=DEV)
    dF0 = torch.empty_like(dL_df)
    lat.backward(dL_df, w, ws, dW, dF0, "bf16")
    assert lat.status() == lbm.LBM_OK
    prm = oracle.params(tau, force_amp=F0, force_mode=m)
    g0 = oracle.stream_push(f0.astype(np.float64))
    L, dth, dg0 = oracle.unroll_grad(g0, steps, prm, thb, utx.astype(np.float64),
                                     uty.astype(np.float64))
    assert abs(float(loss.item()) / L - 1) <= 1e-3
    dWg = _np(dW)

    def rel_l2(a, b):
        return float(np.linalg.norm(a - b) / np.linalg.norm(b))

    tol = 5e-2
    blocks = ((0, 576), (576, 640), (640, 4736), (4736, 4800), (4800, 5376), (5376, 5385))
    errs = [rel_l2(dWg[lo:hi], dth[lo:hi]) for lo, hi in blocks]
    df0 = oracle.stream_pull(dg0)
    msg = (f"{nx}x{ny}x{B} {steps} steps, record {record}: relative L2 error overall "
           f"{rel_l2(dWg, dth):.4e}, per block {['%.2e' % e for e in errs]}, "
           f"dL/df0 {rel_l2(_np(dF0), df0):.4e}")
    print(msg)
    assert rel_l2(dWg, dth) <= tol, msg
    assert max(errs) <= 2.5 * tol, msg  # a wrong block would be off by O(1)
    assert float(dWg @ dth / (np.linalg.norm(dWg) * np.linalg.norm(dth))) >= 0.995, msg
    assert rel_l2(_np(dF0), df0) <= tol, msg
    # deterministic
    dW2 = torch.empty_like(dW)
    lat.backward(dL_df, w, ws, dW2, None, "bf16")
    assert torch.equal(dW, dW2)


@pytest.mark.parametrize("pair", ["f32", "bf16"])
def test_checkpoint_interval_changes_no_bits(lbm, pair):
    """The record copies the start state once, has every later checkpoint
    written by the step that produces it and keeps the last segment's states
    where the backward would recompute them; the backward recomputes the other
    segments from their checkpoints with the same kernel.  Every state the
    adjoint sees is therefore the same bits for any interval k, and so are the
    final state, the loss, dtheta and dL/df0 (n = 5: k = 2 and 3 leave a
    ragged last segment, k = 5 and 8 record only the start).  A second backward
    (whose last segment, for k = 3, has been overwritten by the first one's
    recompute of the other segment) gives the same bits again."""
    nx, ny, B, n = 200, 24, 2, 5
    theta = inputs.xavier_mlp(7, bias_scale=0.3, gain=3.0, out_scale=0.01)
    f0 = _dev(population_field(B, ny, nx, seed=91, neq=0.05))
    utx = _dev(inputs.noise((B, ny, nx), 92, 0.03))
    uty = _dev(inputs.noise((B, ny, nx), 93, 0.03))
    kind = "mlp_f32" if pair == "f32" else "mlp_bf16"
    lat = lbm.Lattice(nx, ny, B, tau=0.6, force_amp=1e-4, force_mode=1, device=DEV)
    w = lbm.weights_struct(_dev(theta))
    lat.set_state(f0)
    lat.step(n, kind, w)
    plain = lat.get_state()
    runs = {}
    for k in (1, 2, 3, 5, 8):
        lat.set_state(f0)
        ws = torch.empty(lat.record_bytes(n, k) // 4, dtype=torch.float32, device=DEV)
        lat.forward_record(n, k, w, ws, pair)
        fin = lat.get_state()
        loss, dL_df = lat.velocity_loss(utx, uty)
        dW = torch.empty(lbm.LBM_MLP_NPARAMS, dtype=torch.float32, device=DEV)
        dF0 = torch.empty_like(dL_df)
        lat.backward(dL_df, w, ws, dW, dF0, pair)
        dW2, dF02 = torch.empty_like(dW), torch.empty_like(dF0)
        lat.backward(dL_df, w, ws, dW2, dF02, pair)
        assert lat.status() == lbm.LBM_OK
        assert torch.equal(dW, dW2) and torch.equal(dF0, dF02), f"k = {k}, second backward"
        # the context's state is the recorded run's end, untouched by the backward
        assert torch.equal(lat.get_state(), fin)
        runs[k] = (fin, loss.clone(), dW, dF0)
    assert torch.equal(runs[1][0], plain)
    assert float(runs[1][2].abs().max()) > 0
    for k in (2, 3, 5, 8):
        for a, b in zip(runs[1], runs[k]):
            assert torch.equal(a, b), f"k = {k}"


@pytest.mark.parametrize("pair", ["f32", "bf16"])
def test_zero_step_record(lbm, pair):
    """An unroll of n = 0 steps: the state is unchanged, dtheta is zero, and
    dL/df0 is dL/df_final (the push of the final adjoint and the pull back
    are inverse permutations, so the bits are kept)."""
    nx, ny, B = 96, 10, 2
    theta = inputs.xavier_mlp(7, bias_scale=0.3, gain=3.0, out_scale=0.01)
    f0 = _dev(population_field(B, ny, nx, seed=95, neq=0.05))
    lat = lbm.Lattice(nx, ny, B, tau=0.6, force_amp=1e-4, force_mode=1, device=DEV)
    w = lbm.weights_struct(_dev(theta))
    lat.set_state(f0)
    before = lat.get_state()
    ws = torch.empty(lat.record_bytes(0, 4) // 4, dtype=torch.float32, device=DEV)
    lat.forward_record(0, 4, w, ws, pair)
    loss, dL_df = lat.velocity_loss(_dev(inputs.noise((B, ny, nx), 96, 0.03)),
                                    _dev(inputs.noise((B, ny, nx), 97, 0.03)))
    dW = torch.full((lbm.LBM_MLP_NPARAMS,), float("nan"), dtype=torch.float32, device=DEV)
    dF0 = torch.empty_like(dL_df)
    lat.backward(dL_df, w, ws, dW, dF0, pair)
    assert lat.status() == lbm.LBM_OK
    assert torch.equal(lat.get_state(), before)
    assert torch.equal(dW, torch.zeros_like(dW))
    assert torch.equal(dF0, dL_df)
