"""GPU parity of the paper's training variant and dataset definition
(SI section 2) against the oracle: losses on a node subset (velocity form and
the population form of Eq. S13) with their gradients, the subsampling filter,
and streaming / anti-streaming of a population field.

Tolerances: the losses are FP64 reductions of per-node errors; the velocity
form takes its moments in FP32 (1e-5 relative on L, 1e-5 of the largest
gradient entry), the population form its differences in FP64 from the FP32
state (1e-12 relative on L before the final FP32 rounding, so 1e-6; gradient
entries are 2 (g - t) rounded once to FP32: 1e-6 relative).  Filter and
streaming move FP32 values: bit-exact.
"""
import numpy as np
import pytest

import oracle
from paper_2403_18466_gb300 import inputs
from gpu_helpers import population_field

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu
DEV = "cuda:0"
_, _, W = oracle.lattice()
W32 = W.astype(np.float32).astype(np.float64)   # the weights the FP32 state is shifted by


@pytest.fixture(scope="module")
def lbm():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_2403_18466_gb300 import lbm as m
    m.load()
    return m


def _dev(a, dtype=torch.float32):
    return torch.tensor(np.ascontiguousarray(a), dtype=dtype, device=DEV)


def _lattice(lbm, nx, ny, B, seed):
    lat = lbm.Lattice(nx, ny, B, device=DEV)
    lat.set_state(_dev(population_field(B, ny, nx, seed=seed, urms=0.04, neq=0.03)))
    return lat


def _post_f64(lat):
    """Post-collision populations g = state + w, formed in FP64 from the raw
    buffer (the state holds g minus the FP32 lattice weights)."""
    st = lat.state_tensor().double().cpu().numpy()
    return st + W32[None, :, None, None]


def _subset(nodes, count, seed, dup=True):
    rng = np.random.default_rng(seed)
    idx = rng.choice(nodes, size=min(count, nodes), replace=False)
    if dup and count > 3:
        idx[-1] = idx[0]          # a repeated node counts twice
        idx[-2] = nodes - 1       # the last node of the last lattice
    return idx.astype(np.int32)


CASES = [(37, 29, 2, 40), (64, 48, 1, 512), (130, 17, 3, 700), (16, 16, 1, 256)]


@pytest.mark.parametrize("nx,ny,B,count", CASES)
def test_velocity_loss_subset_parity(lbm, nx, ny, B, count):
    lat = _lattice(lbm, nx, ny, B, 31)
    idx = _subset(B * nx * ny, count, 32)
    utx, uty = inputs.noise((B, ny, nx), 33, 0.03), inputs.noise((B, ny, nx), 34, 0.03)
    loss, g = lat.velocity_loss_subset(_dev(idx, torch.int32), _dev(utx), _dev(uty))
    L, G = oracle.velocity_loss_subset(lat.get_state().double().cpu().numpy(), idx, utx, uty)
    assert abs(loss.item() / L - 1) <= 1e-5
    G_gpu = g.double().cpu().numpy()
    assert np.abs(G_gpu - G).max() <= 1e-5 * np.abs(G).max()
    assert np.all(G_gpu[G == 0] == 0)
    assert lat.status() == lbm.LBM_OK


@pytest.mark.parametrize("nx,ny,B,count", CASES)
def test_population_loss_subset_parity(lbm, nx, ny, B, count):
    lat = _lattice(lbm, nx, ny, B, 41)
    idx = _subset(B * nx * ny, count, 42)
    gpost = _post_f64(lat)
    target = (gpost + inputs.noise(gpost.shape, 43, 1e-3)).astype(np.float32)
    loss, g = lat.population_loss_subset(_dev(idx, torch.int32), _dev(target))
    L, dLdg = oracle.population_loss_subset(gpost, idx, target.astype(np.float64))
    assert abs(loss.item() / L - 1) <= 1e-6
    # the gradient of g_i(x) is stored where g_i(x) streams to: dL/df = pull(dL/dg)
    G = oracle.stream_pull(dLdg)
    G_gpu = g.double().cpu().numpy()
    assert np.allclose(G_gpu, G, rtol=1e-6, atol=1e-7 * np.abs(G).max())
    assert np.all(G_gpu[G == 0] == 0)


def test_subset_losses_over_all_nodes_match_full_field_forms(lbm):
    nx, ny, B = 48, 40, 2
    lat = _lattice(lbm, nx, ny, B, 51)
    utx, uty = _dev(inputs.noise((B, ny, nx), 52, 0.03)), _dev(inputs.noise((B, ny, nx), 53, 0.03))
    every = torch.arange(B * nx * ny, dtype=torch.int32, device=DEV)
    ls, gs = lat.velocity_loss_subset(every, utx, uty)
    lf, gf = lat.velocity_loss(utx, uty)
    assert abs(ls.item() / lf.item() - 1) <= 1e-5
    assert (gs - gf).abs().max().item() <= 1e-6 * gf.abs().max().item()


def test_subset_loss_argument_errors(lbm):
    lat = _lattice(lbm, 32, 32, 1, 61)
    f = lat.get_state()
    utx = torch.zeros((1, 32, 32), device=DEV)
    empty = torch.zeros(0, dtype=torch.int32, device=DEV)
    with pytest.raises(lbm.LbmError):
        lat.velocity_loss_subset(empty, utx, utx)
    with pytest.raises(lbm.LbmError):
        lat.population_loss_subset(torch.zeros(32 * 32 + 1, dtype=torch.int32, device=DEV), f)
    # an out-of-range index is skipped on the device and reported by lbm_status
    bad = _dev(np.array([3, 32 * 32, -1, 7], dtype=np.int32), torch.int32)
    loss, _ = lat.population_loss_subset(bad, f)
    assert lat.status() == lbm.LBM_ERR_ARG
    lat.clear_status()
    assert lat.status() == lbm.LBM_OK
    ok = _dev(np.array([3, 7], dtype=np.int32), torch.int32)
    loss_ok, _ = lat.population_loss_subset(ok, f)
    assert loss.item() == loss_ok.item()


@pytest.mark.parametrize("nx,ny,B,cg", [(64, 48, 2, 8), (36, 20, 1, 4), (9, 6, 1, 3), (8, 8, 1, 1)])
def test_subsample_parity(lbm, nx, ny, B, cg):
    lat = _lattice(lbm, nx, ny, B, 71)
    got = lat.subsample(cg).cpu().numpy()
    f = lat.get_state().cpu().numpy()
    assert np.array_equal(got, f[:, :, ::cg, ::cg])
    assert np.array_equal(got.astype(np.float64), oracle.subsample(f.astype(np.float64), cg))
    with pytest.raises(lbm.LbmError):
        lat.subsample(5 if nx % 5 else 7)


@pytest.mark.parametrize("nx,ny,B", [(37, 29, 2), (64, 64, 1), (2, 3, 1)])
def test_stream_and_antistream_parity(lbm, nx, ny, B):
    lat = lbm.Lattice(nx, ny, B, device=DEV)
    f = population_field(B, ny, nx, seed=81)
    fd = _dev(f)
    s = lat.stream(fd, 1).cpu().numpy()
    a = lat.stream(fd, -1).cpu().numpy()
    f32 = fd.cpu().numpy().astype(np.float64)
    assert np.array_equal(s.astype(np.float64), oracle.stream_pull(f32))
    assert np.array_equal(a.astype(np.float64), oracle.stream_push(f32))
    assert torch.equal(lat.stream(lat.stream(fd, 1), -1), fd)
    with pytest.raises(lbm.LbmError):
        lat.stream(fd, 0)
    with pytest.raises(lbm.LbmError):
        lat.stream(fd, 1, out=fd)
