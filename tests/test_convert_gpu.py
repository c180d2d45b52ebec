"""The integer-pipe FP32 <-> FP64 conversions of the mixed-precision DP equal the
conversion instructions bit for bit (round to nearest even; zeros, subnormals,
infinities and NaNs included)."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from paper_2507_12349_b300 import binding as B

pytestmark = pytest.mark.gpu


def test_narrow_and_widen_bitwise():
    rng = np.random.default_rng(0)
    x64 = np.concatenate([
        rng.standard_normal(200_000) * np.exp(rng.uniform(-80, 80, 200_000)),      # spans the float range
        np.exp(rng.uniform(-750, 710, 50_000)) * rng.choice([-1, 1], 50_000),      # beyond it: subnormal / inf
        np.array([0.0, -0.0, np.inf, -np.inf, np.nan, 1.0, 3.4028234663852886e38, 3.4028235677973366e38,
                  1.1754943508222875e-38, 1.401298464324817e-45, 7.006492321624085e-46]),
    ])
    # exact ties: a float with its last bit set, plus half an ulp
    f = rng.standard_normal(20_000).astype(np.float32)
    ties = f.astype(np.float64) + np.spacing(f).astype(np.float64) / 2
    x64 = np.concatenate([x64, ties])
    bits32 = rng.integers(0, 2 ** 32, size=x64.size, dtype=np.uint64).astype(np.uint32)
    x32 = bits32.view(np.float32)
    x32[:8] = np.array([0.0, -0.0, np.inf, -np.inf, np.nan, 1e-45, -1e-40, 3.4e38], dtype=np.float32)
    d64 = torch.tensor(x64, device="cuda")
    d32 = torch.tensor(x32, device="cuda")
    narrowed = torch.empty(x64.size, dtype=torch.float32, device="cuda")
    widened = torch.empty(x64.size, dtype=torch.float64, device="cuda")
    B.convert_check(d64, d32, narrowed, widened)
    torch.cuda.synchronize()
    ref_n = d64.to(torch.float32)
    ref_w = d32.to(torch.float64)
    nan_n = torch.isnan(ref_n)
    assert torch.equal(torch.isnan(narrowed), nan_n)
    assert torch.equal(narrowed[~nan_n].view(torch.int32), ref_n[~nan_n].view(torch.int32))
    nan_w = torch.isnan(ref_w)
    assert torch.equal(torch.isnan(widened), nan_w)
    assert torch.equal(widened[~nan_w].view(torch.int64), ref_w[~nan_w].view(torch.int64))
