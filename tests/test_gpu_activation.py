"""GPU accuracy of the tensor-core step's hidden-layer activation (tanh of the
Eq. S10 network), through lbm_activation, against CUDA's tanhf (torch.tanh on
the device) and against float64 tanh:

* the FMA-pipe form y P(min(y^2, 1)), y = a/4, before its bf16 rounding, is
  within half a bf16 ulp of tanh(a) for every input: all finite bf16 values
  of magnitude up to 64, a dense float32 sweep of [-6, 6] and tiny inputs;
* as stored (rounded to bf16, clamped to [-1, 1]) it is exactly the bf16
  rounding of that value, so within one bf16 ulp of tanh;
* the XU form (bf16 input, tanh.approx.bf16x2) is reported and bounded.
"""
import numpy as np
import pytest

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


def _inputs():
    bits = np.arange(0, 1 << 15, dtype=np.uint32)  # all non-negative bf16 patterns
    vals = (bits << 16).view(np.float32)
    vals = vals[np.isfinite(vals) & (vals <= 64.0)]
    dense = np.linspace(-6.0, 6.0, 4_000_001, dtype=np.float32)
    tiny = np.geomspace(1e-30, 1e-2, 20001).astype(np.float32)
    a = np.concatenate([vals, -vals, dense, tiny, -tiny, np.float32([0.0, 4.0, -4.0, 3.9999])])
    return torch.tensor(a, device=DEV)


def _half_ulp_bf16(t):
    """Half a bf16 ulp of |t| (bf16 keeps 8 significant bits)."""
    t = np.abs(t)
    e = np.floor(np.log2(np.where(t > 0, t, 1.0)))
    return np.where(t > 0, 2.0 ** (e - 8), 0.0)


def _bf16_rn(x):
    return torch.tensor(x, dtype=torch.float32).to(torch.bfloat16).float().numpy()


def test_fma_form_within_half_bf16_ulp_of_tanhf(lbm):
    a = _inputs()
    ref_cuda = torch.tanh(a).double().cpu().numpy()     # CUDA tanhf
    ref64 = np.tanh(a.double().cpu().numpy())
    pre = lbm.activation(a, 2).double().cpu().numpy()
    for ref, name in ((ref_cuda, "tanhf"), (ref64, "float64 tanh")):
        hu = _half_ulp_bf16(ref)
        zero = ref == 0
        worst = float(np.max(np.abs(pre[~zero] - ref[~zero]) / hu[~zero]))
        print(f"FMA form before rounding vs {name}: max error {worst:.3f} half-ulps")
        assert worst <= 1.0, worst
        assert np.all(pre[zero] == 0.0)


def test_fma_form_as_stored_is_the_bf16_rounding(lbm):
    """Stored = a bf16 value within half a bf16 ulp of the unrounded value
    (round to nearest; either way on exact ties), clamped to [-1, 1]."""
    a = _inputs()
    pre = lbm.activation(a, 2).cpu().numpy()
    stored = lbm.activation(a, 1).cpu().numpy()
    assert np.array_equal(stored, _bf16_rn(stored))  # representable in bf16
    assert np.all(np.abs(stored.astype(np.float64) - pre) <= _half_ulp_bf16(pre))
    assert np.mean(stored == _bf16_rn(pre)) > 0.999
    ref = np.tanh(a.double().cpu().numpy())
    ulp = 2 * _half_ulp_bf16(ref)
    nz = ref != 0
    worst = float(np.max(np.abs(stored[nz] - ref[nz]) / ulp[nz]))
    print(f"FMA form as stored: max error {worst:.3f} bf16 ulps")
    assert worst <= 1.0
    assert np.all(np.abs(stored) <= 1.0)


def test_xu_form_accuracy(lbm):
    a = _inputs()
    xu = lbm.activation(a, 0).double().cpu().numpy()
    ref = np.tanh(a.double().cpu().numpy())
    nz = np.abs(ref) > 1e-30
    rel = np.abs(xu[nz] - ref[nz]) / np.abs(ref[nz])
    print(f"XU form (bf16 input, tanh.approx.bf16x2): max relative error {rel.max():.3e}")
    assert rel.max() <= 2.0 ** -6
