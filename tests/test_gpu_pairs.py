"""The mixed path's level conversions (mol_pair_split / mol_pair_join),
bit for bit against CUDA's own float64 -> float32 conversion and float64
addition (through torch), over magnitudes that cover every branch of the
integer rounding: float32-normal results (ties, carries into the exponent,
the largest finite values), results that overflow to infinity, float32
subnormal results and underflow to zero, float64 subnormal inputs, signed
zeros, infinities and NaNs, low parts far below the high part; both the
16-byte vectorised kernels and the scalar ones (an unaligned view), and
ragged lengths."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from paper_1308_3214_gb300 import molt

pytestmark = pytest.mark.gpu


def special_values():
    f32max = float(np.finfo(np.float32).max)
    tiny32 = float(np.finfo(np.float32).tiny)
    vals = [0.0, -0.0, 1.0, -1.0, f32max, -f32max, f32max * (1 + 2.0 ** -25), f32max * (1 + 2.0 ** -24),
            f32max * 2, tiny32, tiny32 / 2, tiny32 * (1 - 2.0 ** -30), 2.0 ** -149, 2.0 ** -150,
            2.0 ** -150 * 1.5, 2.0 ** -151, 1e-300, 5e-324, -5e-324, float("inf"), -float("inf"), float("nan"),
            1 + 2.0 ** -24, 1 + 3 * 2.0 ** -24, 1 + 2.0 ** -24 + 2.0 ** -50, 1 - 2.0 ** -25, 2.0 ** 127 * (2 - 2.0 ** -24)]
    return np.array(vals, dtype=np.float64)


def inputs(n, seed):
    rng = np.random.default_rng(seed)
    mant = rng.uniform(-2.0, 2.0, size=n)
    expo = rng.integers(-160, 140, size=n)
    x = np.ldexp(mant, expo)
    # exact ties of the float32 rounding: a float32 value plus half its ulp
    h = rng.uniform(1.0, 2.0, size=n // 8).astype(np.float32).astype(np.float64)
    x[: n // 8] = h + np.ldexp(1.0, -24) * np.sign(rng.uniform(-1, 1, size=n // 8))
    # values a few units of the last float64 place away from a float32: small
    # residuals, whose low part has few bits and lies far below the high part
    k = n // 8
    h = np.ldexp(rng.uniform(-2.0, 2.0, size=k), rng.integers(-140, 120, size=k)).astype(np.float32).astype(np.float64)
    x[k: 2 * k] = h + np.ldexp(rng.integers(-1000, 1000, size=k).astype(np.float64), np.frexp(h)[1] - 53)
    # magnitudes below the float32 normal range down to float64 subnormals
    x[2 * k: 3 * k] = np.ldexp(rng.uniform(-2.0, 2.0, size=k), rng.integers(-1080, -100, size=k))
    return np.concatenate([x, special_values()])


def same_bits(a, b):
    """Equal encodings, any NaN equal to any NaN."""
    ib = torch.int32 if a.dtype == torch.float32 else torch.int64
    return bool(((a.view(ib) == b.view(ib)) | (torch.isnan(a) & torch.isnan(b))).all())


def check(xd):
    hi, lo = molt.pair_split(xd)
    rhi = xd.float()
    assert same_bits(hi, rhi)
    finite = torch.isfinite(xd) & torch.isfinite(rhi)
    assert same_bits(lo[finite], (xd[finite] - rhi[finite].double()).float())
    assert same_bits(molt.pair_join(hi, lo), hi.double() + lo.double())


@pytest.mark.parametrize("n", [4096, 4099, 1_000_003])
def test_pair_conversions_bitwise(n):
    x = torch.from_numpy(inputs(n, 7 + n)).cuda()
    check(x)                        # 16-byte aligned: the vectorised kernels
    buf = torch.empty(x.numel() + 1, dtype=torch.float64, device="cuda")
    buf[1:] = x
    xs = buf[1:]                    # an 8-byte offset: the scalar kernels
    hi = torch.empty(x.numel() + 1, dtype=torch.float32, device="cuda")[1:]
    lo = torch.empty(x.numel() + 1, dtype=torch.float32, device="cuda")[1:]
    molt.pair_split(xs, hi, lo)
    assert same_bits(hi, x.float())
    finite = torch.isfinite(x) & torch.isfinite(x.float())
    assert same_bits(lo[finite], (x[finite] - x.float()[finite].double()).float())
    out = torch.empty(x.numel() + 1, dtype=torch.float64, device="cuda")[1:]
    molt.pair_join(hi, lo, out)
    assert same_bits(out, hi.double() + lo.double())


def test_pair_join_arbitrary_pairs():
    """mol_pair_join on pairs that no split produced: random encodings, and
    normal pairs with every exponent gap from 0 to 60 in either order."""
    rng = np.random.default_rng(11)
    n = 1 << 20
    bits = rng.integers(0, 1 << 32, size=(2, n), dtype=np.uint64).astype(np.uint32)
    hi = torch.from_numpy(bits[0].view(np.float32).copy()).cuda()
    lo = torch.from_numpy(bits[1].view(np.float32).copy()).cuda()
    assert same_bits(molt.pair_join(hi, lo), hi.double() + lo.double())
    e = rng.integers(-100, 100, size=n)
    h = np.ldexp(rng.uniform(-2.0, 2.0, size=n), e).astype(np.float32)
    l = np.ldexp(rng.uniform(-2.0, 2.0, size=n), e - rng.integers(-4, 61, size=n)).astype(np.float32)
    hi, lo = torch.from_numpy(h).cuda(), torch.from_numpy(l).cuda()
    assert same_bits(molt.pair_join(hi, lo), hi.double() + lo.double())


def test_pair_conversions_reject_bad_arguments():
    x = torch.zeros(8, dtype=torch.float64, device="cuda")
    with pytest.raises(TypeError):
        molt.pair_split(x.float())
    with pytest.raises(ValueError):
        molt.pair_split(x, torch.zeros(4, device="cuda"), torch.zeros(8, device="cuda"))
