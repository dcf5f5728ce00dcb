"""The 32-bit fixed-point conversions of the histogram flushes equal CUDA's
64-bit conversions bit for bit (round to nearest, ties to even).

float -> 64-bit integer over [0, 2^64): zero, subnormals, halves (ties),
values next to the 2^23, 2^24, 2^32 and 2^48 boundaries, the largest floats
below 2^64, and log-uniform random values.  Word pair (hi, lo) -> float of
hi 2^24 + lo over hi <= 256 (2^24 - 1), lo < 2^32: sums on both sides of
2^48 (where the carry of lo's top byte decides the path), exact ties at
every binade, and random pairs.  The exact nearest float is also checked on
the host for the pairs, from the integer sum."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def nearest_f32(h: int) -> np.float32:
    """Nearest float32 to the integer h (ties to even), exactly."""
    if h == 0:
        return np.float32(0.0)
    e = h.bit_length() - 24           # drop e low bits
    if e <= 0:
        return np.float32(h)
    q, r = divmod(h, 1 << e)
    half = 1 << (e - 1)
    if r > half or (r == half and q & 1):
        q += 1
    return np.float32(np.ldexp(np.float64(q), e))


def floats_to_test(rng):
    vals = [0.0, 1e-45, 1e-38, 0.25, 0.5, 1.0, 1.5, 2.5, 3.5, 0.49999997, 0.50000006,
            2.0 ** 23 - 0.5, 2.0 ** 23, 2.0 ** 23 + 1, 2.0 ** 24 - 1, 2.0 ** 24, 2.0 ** 24 + 2,
            2.0 ** 31, 2.0 ** 32 - 256, 2.0 ** 32, 2.0 ** 32 + 512, 2.0 ** 47, 2.0 ** 48,
            2.0 ** 56, 2.0 ** 63, float(np.nextafter(np.float32(2.0 ** 64), np.float32(0)))]
    v = np.array(vals, np.float32)
    halves = (rng.integers(0, 1 << 22, 4000) + 0.5).astype(np.float32)
    logu = np.exp2(rng.uniform(-20, 63.99, 200000)).astype(np.float32)
    near32 = np.float32(2.0 ** 32) - rng.integers(0, 200, 2000).astype(np.float32) * 256
    v = np.concatenate([v, halves, logu, near32]).astype(np.float32)
    assert (v >= 0).all() and (v.astype(np.float64) < 2.0 ** 64).all()
    return v


def pairs_to_test(rng):
    hmax = 256 * ((1 << 24) - 1)
    hi = [0, 0, 1, (1 << 24) - 1, (1 << 24) - 1, 1 << 24, hmax, hmax, 12345]
    lo = [0, (1 << 32) - 1, 0, (1 << 24) - 1, 1 << 24, 0, 0, (1 << 32) - 1, (1 << 31) + 7]
    n = 100000
    h = list(rng.integers(0, hmax + 1, n, dtype=np.int64))
    l = list(rng.integers(0, 1 << 32, n, dtype=np.int64))
    # small hi: the sum is near 2^48 only through lo's carry
    h += list(rng.integers((1 << 24) - 300, 1 << 24, 20000, dtype=np.int64))
    l += list(rng.integers(0, 1 << 32, 20000, dtype=np.int64))
    # exact ties: sums (2q + 1) 2^(e-1) with e low bits dropped
    for e in range(1, 33):
        for _ in range(200):
            top = int(rng.integers(1 << 23, 1 << 24))
            s = (top << e) + (1 << (e - 1))
            if s >= (hmax << 24):
                continue
            hh = min(s >> 24, hmax)
            hi.append(hh); lo.append(s - (hh << 24))
    hi = np.array(hi + h, np.int64)
    lo = np.array(lo + l, np.int64)
    ok = (lo < (1 << 32)) & (hi <= hmax) & (lo >= 0) & (hi >= 0)
    return hi[ok], lo[ok]


def test_fixed_point_conversions_match_cuda():
    import paper_1804_05061_b300 as eng
    rng = np.random.default_rng(7)
    v = floats_to_test(rng)
    hi, lo = pairs_to_test(rng)
    vt = torch.from_numpy(v).cuda()
    hit = torch.from_numpy(hi.astype(np.uint32).view(np.int32)).cuda()
    lot = torch.from_numpy(lo.astype(np.uint32).view(np.int32)).cuda()
    fx, fl = eng.debug_fixed_point(vt, hit, lot)
    rfx, rfl = eng.debug_fixed_point(vt, hit, lot, reference=True)
    fx, rfx = fx.cpu().numpy().view(np.uint64), rfx.cpu().numpy().view(np.uint64)
    bad = np.nonzero(fx != rfx)[0]
    assert bad.size == 0, [(float(v[i]), int(fx[i]), int(rfx[i])) for i in bad[:5]]
    fl, rfl = fl.cpu().numpy(), rfl.cpu().numpy()
    bad = np.nonzero(fl.view(np.uint32) != rfl.view(np.uint32))[0]
    assert bad.size == 0, [(int(hi[i]), int(lo[i]), float(fl[i]), float(rfl[i])) for i in bad[:5]]
    # the integer side on the host: nearest integer, ties to even
    for i in list(range(40)) + list(rng.integers(0, v.size, 3000)):
        x = float(v[i])
        q = int(np.floor(x)); r = x - q
        if r > 0.5 or (r == 0.5 and q & 1):
            q += 1
        assert int(fx[i]) == q, (x, int(fx[i]), q)
    # the float side on the host: exact nearest float of the integer sum
    for i in list(range(9)) + list(rng.integers(0, hi.size, 3000)):
        s = (int(hi[i]) << 24) + int(lo[i])
        assert fl[i] == nearest_f32(s), (int(hi[i]), int(lo[i]), float(fl[i]), nearest_f32(s))
