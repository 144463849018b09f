"""The 16-bit storage codec behind the C ABI (vlasov_encode / vlasov_decode).

The codes and scales the library writes are compared bit for bit with a numpy
restatement of the documented encode: w = the value rounded to FP32, scale = the
line's largest w (at least 2^-64 for BF16 codes, 0 for an empty FP16 line), code =
the IEEE FP32 quotient w / scale rounded to nearest even in BF16 or FP16 (0 where the
scale is 0).  Decoding must give code x scale exactly in FP64 and that product rounded
to nearest in FP32.  Lines of every length the storage takes (16, 24, 32, 40, 48) and a
few others, FP64 and FP32 sources, lines that are all zero and lines far below 2^-64
are covered.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TDT = {"bf16": torch.bfloat16, "f16": torch.float16}


def _rn_bf16_bits(q32):
    # round to nearest even of FP32 values into BF16, on the bit patterns
    b = q32.view(np.uint32).astype(np.uint64)
    return ((b + 0x7FFF + ((b >> 16) & 1)) >> 16).astype(np.uint16)


def _expected(v, fmt):
    w = v.astype(np.float32)
    m = np.maximum(w.max(axis=-1), np.float32(0))
    if fmt == "bf16":
        m = np.maximum(m, np.float32(2.0 ** -64))
    with np.errstate(divide="ignore", invalid="ignore"):
        q = np.where(m[..., None] > 0, w / m[..., None], np.float32(0)).astype(np.float32)
    codes = _rn_bf16_bits(q) if fmt == "bf16" else q.astype(np.float16).view(np.uint16)
    return codes, m.astype(np.float32)


def _values(nlines, nuz, seed):
    rng = np.random.default_rng(seed)
    v = rng.random((nlines, nuz)) ** 3 * np.exp(rng.uniform(-20, 5, size=(nlines, 1)))
    v[rng.random((nlines, nuz)) < 0.05] = 0.0
    v[3] = 0.0                  # an empty line
    v[5] *= 2.0 ** -90          # a line whose largest value lies far below 2^-64
    v[7, :] = 1.0               # a constant line: every code is 1
    return v


@pytest.mark.parametrize("fmt", ["bf16", "f16"])
@pytest.mark.parametrize("src", ["f64", "f32"])
@pytest.mark.parametrize("nuz", [16, 24, 32, 40, 48, 4, 12, 100, 128])
def test_encode_matches_restatement_bit_for_bit(fmt, src, nuz):
    from paper_2110_15867_gb300 import binding as B
    B.load()
    nlines = 1037  # not a multiple of any number of lines per warp
    v = _values(nlines, nuz, seed=nuz)
    if src == "f32":
        v = v.astype(np.float32)
    codes, scale = B.encode_lines(torch.from_numpy(v).cuda(), TDT[fmt])
    torch.cuda.synchronize()
    want_c, want_s = _expected(v, fmt)
    got_c = codes.view(torch.int16).cpu().numpy().view(np.uint16)
    got_s = scale.cpu().numpy()
    assert np.array_equal(got_s.view(np.uint32), want_s.view(np.uint32))
    assert np.array_equal(got_c, want_c)


@pytest.mark.parametrize("fmt", ["bf16", "f16"])
def test_decode_is_code_times_scale(fmt):
    from paper_2110_15867_gb300 import binding as B
    B.load()
    v = _values(517, 32, seed=3)
    codes, scale = B.encode_lines(torch.from_numpy(v).cuda(), TDT[fmt])
    c = codes.to(torch.float64).cpu().numpy()
    s = scale.cpu().numpy().astype(np.float64)
    exact = c * s[:, None]
    d64 = B.decode_lines(codes, scale).cpu().numpy()
    d32 = B.decode_lines(codes, scale, torch.float32).cpu().numpy()
    assert np.array_equal(d64, exact)
    assert np.array_equal(d32, exact.astype(np.float32))
    # the encode round trip: each value within half a unit in the last place of its code
    # (relative to the line scale) once the scale is at least the BF16 floor
    ulp = 2.0 ** -8 if fmt == "bf16" else 2.0 ** -11
    big = s >= 2.0 ** -60
    err = np.abs(d64 - v)[big]
    assert (err <= ulp * s[big][:, None] * (1 + 1e-6) + 2.0 ** -24 * np.abs(v[big])).all()


def test_encode_a_whole_grid_in_slabs_equals_one_call():
    # a slab of x-planes is a contiguous run of u_z lines: encoding slab by slab into
    # views of one array gives the same codes as one call over the grid
    from paper_2110_15867_gb300 import binding as B
    B.load()
    rng = np.random.default_rng(5)
    f = torch.from_numpy(rng.random((4, 3, 2, 8, 8, 16))).cuda()
    c1, s1 = B.encode_lines(f, torch.bfloat16)
    c2 = torch.empty_like(c1)
    s2 = torch.empty_like(s1)
    for ix in range(4):
        B.encode_lines(f[ix], torch.bfloat16, codes=c2[ix], scale=s2[ix])
    torch.cuda.synchronize()
    assert torch.equal(c1.view(torch.int16), c2.view(torch.int16)) and torch.equal(s1, s2)
