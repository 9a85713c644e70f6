"""The FP32 facts the split-precision kernels rely on, checked on the host in
IEEE single precision (NumPy float32 rounds to nearest even, as the packed
FP32 instructions of the kernels do).

* Slicing: x with |x| < 2^8 is cut into q_0 = rint(x), then q_i = rint of the
  remainder times 256; |q_0| <= 256, |q_i| <= 128, and every q_i * 2^-8i is
  a BF16 number (8 significant bits).
* rint by the shift 1.5 * 2^23: (x + M) - M equals rint(x) for |x| < 2^22.
* The chunk split of the drain: level 0 of a 192-K chunk is an integer of
  magnitude <= 192 * 2^16, level 1 a multiple of 2^-8 of magnitude
  <= 192 * 2 * 256 * 128 * 2^-8; with r = rint(y1), x0 + r and y1 - r are
  exact, so the pair holds x0 + y1 exactly.
* The biased drain exponent byte b = 127 + d placed in the FP32 exponent
  field is 2^d for d in [-126, 0], and b = 0 gives the factor 0.
"""
import numpy as np

F = np.float32
M = F(12582912.0)  # 1.5 * 2^23


def slices(x, S):
    """Slices of float32 values x (|x| < 2^8) as the slab kernels cut them
    (single float here; the kernels carry a float-float remainder)."""
    out = []
    y = x.astype(np.float32)
    for i in range(S):
        q = np.rint(y).astype(np.float32)
        out.append(q)
        y = ((y - q) * F(256.0)).astype(np.float32)
    return out


def test_slice_ranges_and_bf16_exactness():
    rng = np.random.default_rng(7)
    x = (rng.uniform(-1, 1, 200_000) * 256).astype(np.float32)
    x = np.clip(x, np.nextafter(F(-256), F(0)), np.nextafter(F(256), F(0)))
    qs = slices(x, 5)
    assert np.abs(qs[0]).max() <= 256
    for q in qs[1:]:
        assert np.abs(q).max() <= 128
    for i, q in enumerate(qs):
        v = (q * F(2.0 ** (-8 * i))).astype(np.float32)
        bits = v.view(np.uint32)
        # BF16 keeps the top 16 bits of the float32 pattern: the low 16 are zero
        assert np.all((bits & 0xFFFF) == 0), i
    # the slices sum back to x up to the last slice's unit
    back = sum(q.astype(np.float64) * 2.0 ** (-8 * i) for i, q in enumerate(qs))
    assert np.abs(back - x.astype(np.float64)).max() <= 0.5 * 2.0 ** (-32) + 2.0 ** -40


def test_rint_by_shift():
    rng = np.random.default_rng(3)
    x = (rng.uniform(-1, 1, 500_000) * 2 ** 21).astype(np.float32)
    halves = (rng.integers(-2 ** 20, 2 ** 20, 10_000) + F(0.5)).astype(np.float32)  # ties go to even
    for v in (x, halves):
        r = ((v + M).astype(np.float32) - M).astype(np.float32)
        assert np.array_equal(r, np.rint(v))


def test_exact_chunk_split():
    rng = np.random.default_rng(11)
    n = 1_000_000
    x0 = rng.integers(-192 * 2 ** 16, 192 * 2 ** 16 + 1, n).astype(np.float32)
    y1max = 192 * 2 * 256 * 128  # in units of 2^-8
    y1 = (rng.integers(-y1max, y1max + 1, n) / 256.0).astype(np.float32)
    assert np.array_equal(y1.astype(np.float64) * 256, np.round(y1.astype(np.float64) * 256))
    r = ((y1 + M).astype(np.float32) - M).astype(np.float32)
    s = (x0 + r).astype(np.float32)
    e = (y1 - r).astype(np.float32)
    assert np.abs(s).max() < 2 ** 24 and np.abs(e).max() <= 0.5
    exact = x0.astype(np.float64) + y1.astype(np.float64)
    assert np.array_equal(s.astype(np.float64) + e.astype(np.float64), exact)
    # extremes of the bounds
    for a, b in ((192 * 2 ** 16, y1max / 256.0), (-192 * 2 ** 16, -y1max / 256.0)):
        a, b = F(a), F(b)
        rr = F(F(b + M) - M)
        assert float(F(a + rr)) + float(F(b - rr)) == float(a) + float(b)


def test_biased_exponent_byte():
    d = np.arange(-126, 1)
    b = (127 + d).astype(np.uint32)
    # the kernels move the byte to bits 24..31 and shift right once
    f = ((b << 24) >> 1).astype(np.uint32).view(np.float32)
    assert np.array_equal(f.astype(np.float64), 2.0 ** d)
    assert ((np.uint32(0) << 24) >> 1).view(np.float32) == 0.0
