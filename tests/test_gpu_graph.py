"""CUDA-graph capture of the library's launch sequences.

Every entry point only enqueues work on the lattice's stream: no host
synchronisation and, once a first call has created the library's scratch
(weight-gradient partial sums) and set its kernels' shared-memory attributes,
no allocation.  So a sequence of calls -- n steps, or a whole unrolled
training step (state in, record, loss, backward) -- can be captured once into
a CUDA graph and replayed; consecutive tensor-core steps keep their
programmatic-dependent-launch edges inside the graph.  The host-side state the
calls keep (the current buffer, the record's layout) is updated at capture
exactly as by a direct call, and every replay runs the same kernels on the
same buffers.  The replays must give the bits of the same calls issued
directly.
"""
import numpy as np
import pytest

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


@pytest.mark.parametrize("kind", ["bgk", "smag", "mlp_f32", "mlp_bf16"])
def test_steps_replayed_from_a_graph(lbm, kind):
    nx, ny, B, n, reps = 200, 40, 2, 6, 3
    f0 = _dev(population_field(B, ny, nx, seed=101, neq=0.02))
    w = lbm.weights_struct(_dev(inputs.xavier_mlp(3, out_scale=0.3)))
    s = torch.cuda.Stream(device=DEV)
    args = dict(tau=0.6, smag_cs=0.1, force_amp=1e-4, force_mode=1, stream=s, device=DEV)
    lat = lbm.Lattice(nx, ny, B, **args)
    ref = lbm.Lattice(nx, ny, B, **args)
    torch.cuda.synchronize()  # inputs and buffers were made on the default stream
    with torch.cuda.stream(s):
        lat.set_state(f0)
        lat.step(2, kind, w)  # first calls: kernel attributes
        lat.set_state(f0)
    torch.cuda.synchronize()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g, stream=s):
        lat.step(n, kind, w)
    with torch.cuda.stream(s):
        for _ in range(reps):
            g.replay()
        ref.set_state(f0)
        ref.step(n * reps, kind, w)
        got, want = lat.get_state(), ref.get_state()
    torch.cuda.synchronize()
    assert lat.status() == lbm.LBM_OK and ref.status() == lbm.LBM_OK
    assert torch.equal(got, want)


@pytest.mark.parametrize("pair", ["f32", "bf16"])
def test_training_step_replayed_from_a_graph(lbm, pair):
    nx, ny, B, n, k = 160, 24, 2, 8, 3
    f0 = _dev(population_field(B, ny, nx, seed=111, neq=0.05))
    utx = _dev(inputs.noise((B, ny, nx), 112, 0.03))
    uty = _dev(inputs.noise((B, ny, nx), 113, 0.03))
    w = lbm.weights_struct(_dev(inputs.xavier_mlp(7, bias_scale=0.3, gain=3.0, out_scale=0.01)))
    s = torch.cuda.Stream(device=DEV)
    lat = lbm.Lattice(nx, ny, B, tau=0.6, force_amp=1e-4, force_mode=1, stream=s, device=DEV)
    ws = torch.empty(lat.record_bytes(n, k) // 4, dtype=torch.float32, device=DEV)
    loss = torch.empty(1, dtype=torch.float32, device=DEV)
    dL = torch.empty(lat.shape, dtype=torch.float32, device=DEV)
    dW = torch.empty(lbm.LBM_MLP_NPARAMS, dtype=torch.float32, device=DEV)
    dF0 = torch.empty_like(dL)
    p = lbm._ptr

    def train_step():
        lat.set_state(f0)
        lat.forward_record(n, k, w, ws, pair)
        lbm._check(lat.lib.lbm_velocity_loss(lat.ctx, p(utx), p(uty), p(loss), p(dL)),
                   "lbm_velocity_loss")
        lat.backward(dL, w, ws, dW, dF0, pair)

    torch.cuda.synchronize()  # inputs and buffers were made on the default stream
    with torch.cuda.stream(s):
        train_step()  # direct call: the reference, and the library's first-use set-up
    torch.cuda.synchronize()
    assert lat.status() == lbm.LBM_OK
    want = [t.clone() for t in (loss, dW, dF0)]
    assert float(want[1].abs().max()) > 0
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g, stream=s):
        train_step()
    for rep in range(2):
        for t in (loss, dW, dF0):
            t.fill_(float("nan"))
        torch.cuda.synchronize()
        with torch.cuda.stream(s):
            g.replay()
        torch.cuda.synchronize()
        for a, b in zip((loss, dW, dF0), want):
            assert torch.equal(a, b), f"replay {rep}"
    assert lat.status() == lbm.LBM_OK
