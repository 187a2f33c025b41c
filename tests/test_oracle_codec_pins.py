"""Pins for the oracle's compression codec (Sec. 7.1, Sec. 8): uniform quantisation of
the coefficients, bits per vertex, and the NMSVE with its geometric Laplacian.

Every check compares the oracle with something computed another way: the
nearest quantiser level found by exhaustive search, exactly representable
grids, the size of the coded payload, geometric Laplacians worked out by hand
on two right triangles, and invariants (translation, scaling, flat regular
grids).  ``test_codec_planted_mistakes_are_caught`` plants slips on the CPU.
"""
import numpy as np
import pytest

from oracle import bsp_oracle as O


def _blocks(seed=0, shapes=((7, 4), (5, 4), (9, 4))):
    rng = np.random.default_rng(seed)
    return [(rng.standard_normal(s) * rng.uniform(0.1, 10.0)).astype(np.float32) for s in shapes]


# --------------------------------------------------------------------------
# quantiser
# --------------------------------------------------------------------------

def check_quantize_nearest_level(O=O):
    """Each code is the nearest of the 2^bits levels (exhaustive search in FP64)."""
    E = _blocks()
    for bits in (1, 2, 5, 12):
        codes, ranges = O.quantize(E, bits)
        q = (1 << bits) - 1
        for Eb, Cb, Rb in zip(E, codes, ranges):
            # the range is the column's extreme values, found by sorting
            srt = np.sort(Eb, axis=0)
            assert np.array_equal(Rb[:, 0], srt[0]) and np.array_equal(Rb[:, 1], srt[-1])
            lo = srt[0].astype(np.float64)
            hi = srt[-1].astype(np.float64)
            levels = lo[None, :] + np.arange(q + 1)[:, None] * ((hi - lo) / q)[None, :]
            for r in range(Eb.shape[0]):
                d = np.abs(Eb[r].astype(np.float64)[None, :] - levels)   # (levels, cols)
                best = np.argmin(d, axis=0)
                srtd = np.sort(d, axis=0)
                step = (hi - lo) / q
                clear = (srtd[1] - srtd[0]) > 1e-4 * step     # not a near tie
                assert np.array_equal(Cb[r][clear], best[clear]), (bits, r)
            # the extremes take the end codes
            cols = np.arange(Eb.shape[1])
            assert np.all(Cb[np.argmin(Eb, axis=0), cols] == 0)
            assert np.all(Cb[np.argmax(Eb, axis=0), cols] == q)


def check_dequantize_error_bound(O=O):
    """|e - e~| <= half a step (plus rounding), and e~ sits on the level of its code."""
    E = _blocks(seed=1)
    for bits in (3, 8, 12):
        codes, ranges = O.quantize(E, bits)
        rec = O.dequantize(codes, ranges, bits, np.float32)
        q = (1 << bits) - 1
        for Eb, Cb, Rb, Xb in zip(E, codes, ranges, rec):
            step = (Rb[:, 1].astype(np.float64) - Rb[:, 0]) / q
            err = np.abs(Xb.astype(np.float64) - Eb)
            assert np.all(err <= 0.5 * step * (1 + 1e-4) + 4 * np.abs(Eb) * 2.0 ** -23)
            lvl = (Xb.astype(np.float64) - Rb[:, 0]) / step
            assert np.allclose(lvl, Cb, atol=1e-3)


def check_quantize_exact_grid(O=O):
    """Values on an exactly representable grid get their grid index and come back bit-exact."""
    bits = 8
    rng = np.random.default_rng(2)
    idx = rng.integers(0, 256, size=(20, 3))
    idx[0] = 0
    idx[1] = 255
    lo = np.float32(-1.5)
    E = [(lo + idx * np.float32(2.0 ** -8)).astype(np.float32)]
    codes, ranges = O.quantize(E, bits)
    assert np.array_equal(codes[0], idx)
    rec = O.dequantize(codes, ranges, bits, np.float32)
    assert np.array_equal(rec[0], E[0])


def test_quantize_nearest_level():
    check_quantize_nearest_level()


def test_dequantize_error_bound():
    check_dequantize_error_bound()


def test_quantize_exact_grid():
    check_quantize_exact_grid()


def test_quantize_degenerate_columns():
    """A constant column codes to 0 and decodes exactly; 1 bit splits at the midpoint; 16 bits
    reach code 65535; float64 coefficients are coded in float64."""
    E = [np.array([[2.5, -1.0], [2.5, 0.0], [2.5, 3.0], [2.5, 0.9], [2.5, 1.1]], np.float32)]
    codes, ranges = O.quantize(E, 1)
    assert np.all(codes[0][:, 0] == 0)
    assert np.array_equal(codes[0][:, 1], [0, 0, 1, 0, 1])   # midpoint 1.0
    rec = O.dequantize(codes, ranges, 1, np.float32)
    assert np.all(rec[0][:, 0] == np.float32(2.5))
    codes16, _ = O.quantize(E, 16)
    assert codes16[0].dtype == np.uint16 and codes16[0][:, 1].max() == 65535
    E64 = [b.astype(np.float64) for b in _blocks(seed=4)]
    c64, r64 = O.quantize(E64, 12)
    assert r64[0].dtype == np.float64
    rec64 = O.dequantize(c64, r64, 12, np.float64)
    for Eb, Xb, Rb in zip(E64, rec64, r64):
        assert np.all(np.abs(Xb - Eb) <= 0.5 * (Rb[:, 1] - Rb[:, 0]) / 4095 * (1 + 1e-9))


def test_bits_per_vertex_counts_the_payload():
    """bpv x n is the number of payload bits: every xyz coefficient coded with q bits."""
    rng = np.random.default_rng(5)
    c_blocks = rng.integers(8, 40, size=11)
    n = 3000
    E = [rng.standard_normal((c, 3)).astype(np.float32) for c in c_blocks]
    for bits in (6, 12):
        codes, _ = O.quantize(E, bits)
        payload_bits = sum(cb.size for cb in codes) * bits
        assert O.bits_per_vertex(c_blocks, n, bits) * n == pytest.approx(payload_bits, rel=1e-15)


# --------------------------------------------------------------------------
# geometric Laplacian and NMSVE
# --------------------------------------------------------------------------

TRI = np.array([[0, 1, 2]])
X345 = np.array([[0.0, 0, 0], [3, 0, 0], [0, 4, 0]])     # sides 3, 4, 5
X51213 = np.array([[0.0, 0, 0], [5, 0, 0], [0, 12, 0]])  # sides 5, 12, 13
# worked by hand: v_i - (sum_j v_j / d_ij) / (sum_j 1 / d_ij)
GL345 = np.array([[-12 / 7, -12 / 7, 0], [3, -1.5, 0], [-4 / 3, 4, 0]])
GL51213 = np.array([[-60 / 17, -60 / 17, 0], [5, -10 / 3, 0], [-12 / 5, 12, 0]])


def flat_grid(N):
    xs, ys = np.meshgrid(np.arange(N, dtype=np.float64), np.arange(N, dtype=np.float64))
    X = np.stack([xs.ravel(), ys.ravel(), np.zeros(N * N)], axis=1)
    f = []
    for i in range(N - 1):
        for j in range(N - 1):
            a, b, c, d = i * N + j, i * N + j + 1, (i + 1) * N + j, (i + 1) * N + j + 1
            f += [[a, b, d], [a, d, c]]
    return X, np.array(f)


def check_gl_hand_values(O=O):
    assert np.allclose(O.geometric_laplacian(X345, TRI), GL345, atol=1e-12)
    assert np.allclose(O.geometric_laplacian(X51213, TRI), GL51213, atol=1e-12)


def check_nmsve_hand_values(O=O):
    """Each GL uses the edge lengths of its own geometry."""
    val, a, g = O.nmsve(X345, X51213, TRI)
    assert a == pytest.approx(np.sqrt(68.0), rel=1e-14)
    assert g == pytest.approx(np.linalg.norm(GL345 - GL51213), rel=1e-13)
    assert val == pytest.approx((a + g) / 6.0, rel=1e-14)


def check_gl_invariants(O=O):
    X, F = flat_grid(7)
    GL = O.geometric_laplacian(X, F)
    interior = [(i * 7 + j) for i in range(1, 6) for j in range(1, 6)]
    assert np.allclose(GL[interior], 0.0, atol=1e-12)      # symmetric neighbour pairs
    rng = np.random.default_rng(6)
    Y = X + 0.2 * rng.standard_normal(X.shape)
    t = np.array([0.3, -1.2, 2.0])
    assert np.allclose(O.geometric_laplacian(Y + t, F), O.geometric_laplacian(Y, F), atol=1e-12)
    assert np.allclose(O.geometric_laplacian(2.5 * Y, F), 2.5 * O.geometric_laplacian(Y, F),
                       atol=1e-12)
    # faces listed twice (shared sides repeat) change nothing
    assert np.allclose(O.geometric_laplacian(Y, np.concatenate([F, F[:, ::-1]])),
                       O.geometric_laplacian(Y, F), atol=1e-14)
    # a translated copy: the GL term vanishes and ||v - v~|| = sqrt(n) |t|
    n = X.shape[0]
    val, a, g = O.nmsve(Y, Y + t, F)
    assert g == pytest.approx(0.0, abs=1e-12)
    assert a == pytest.approx(np.sqrt(n) * np.linalg.norm(t), rel=1e-13)
    assert val == pytest.approx(a / (2 * n), rel=1e-12)
    # a scaled copy: ||GL(v) - GL(s v)|| = |1 - s| ||GL(v)||
    _, _, g = O.nmsve(Y, 0.75 * Y, F)
    assert g == pytest.approx(0.25 * np.linalg.norm(O.geometric_laplacian(Y, F)), rel=1e-12)
    assert O.nmsve(Y, Y, F)[0] == 0.0


def test_gl_hand_values():
    check_gl_hand_values()


def test_nmsve_hand_values():
    check_nmsve_hand_values()


def test_gl_invariants():
    check_gl_invariants()


def test_gl_isolated_and_coincident_vertices():
    """A vertex without faces keeps GL = v; a neighbour at distance 0 carries no weight."""
    X = np.array([[0.0, 0, 0], [3, 0, 0], [0, 4, 0], [7, 7, 7]])
    GL = O.geometric_laplacian(X, TRI)
    assert np.allclose(GL[:3], GL345) and np.array_equal(GL[3], X[3])
    Xc = np.array([[0.0, 0, 0], [0, 0, 0], [0, 4, 0]])     # vertices 0 and 1 coincide
    GLc = O.geometric_laplacian(Xc, TRI)
    # 0 and 1 see only vertex 2 (their mutual edge has no length): GL = v - v_2
    assert np.allclose(GLc[0], [0, -4, 0]) and np.allclose(GLc[1], [0, -4, 0])
    assert np.allclose(GLc[2], [0, 4, 0])                   # mean of two coincident points


# --------------------------------------------------------------------------
# planted mistakes
# --------------------------------------------------------------------------

class _Mutant:
    def __init__(self, **over):
        self.__dict__.update({k: getattr(O, k) for k in dir(O) if not k.startswith("__")})
        self.__dict__.update(over)


def test_codec_planted_mistakes_are_caught():
    def quantize_floor(E, bits):
        codes, ranges = O.quantize(E, bits)
        out = []
        for Eb, Rb in zip(E, ranges):
            q = np.float32((1 << bits) - 1)
            s = q / (Rb[:, 1] - Rb[:, 0])
            out.append(np.clip(np.floor((Eb - Rb[:, 0]) * s), 0, q).astype(np.uint16))
        return out, ranges

    def quantize_block_range(E, bits):      # one range per block instead of per column
        codes, ranges = [], []
        for Eb in E:
            lo, hi = Eb.min(), Eb.max()
            q = np.float32((1 << bits) - 1)
            codes.append(np.clip(np.rint((Eb - lo) * (q / (hi - lo))), 0, q).astype(np.uint16))
            ranges.append(np.stack([np.full(Eb.shape[1], lo), np.full(Eb.shape[1], hi)], 1))
        return codes, ranges

    def dequantize_off_by_one(codes, ranges, bits, dtype=np.float32):
        return O.dequantize(codes, ranges, bits + 1, dtype) if bits < 16 else codes

    def gl_length_weights(X, faces):         # weights d instead of 1 / d
        X = np.asarray(X, float)
        num = np.zeros_like(X)
        den = np.zeros(len(X))
        for a, b in O.undirected_edges(faces=faces):
            d = np.linalg.norm(X[a] - X[b])
            num[a] += X[b] * d
            den[a] += d
            num[b] += X[a] * d
            den[b] += d
        return X - num / np.maximum(den, 1e-300)[:, None]

    def gl_no_dedupe(X, faces):              # every face side counted, shared sides twice
        X = np.asarray(X, float)
        f = np.asarray(faces)
        e = np.concatenate([f[:, [0, 1]], f[:, [1, 2]], f[:, [2, 0]]])
        num = np.zeros_like(X)
        den = np.zeros(len(X))
        for a, b in e:
            d = np.linalg.norm(X[a] - X[b])
            num[a] += X[b] / d
            den[a] += 1 / d
            num[b] += X[a] / d
            den[b] += 1 / d
        return X - num / den[:, None]

    def nmsve_squared(X, Xr, faces):
        val, a, g = O.nmsve(X, Xr, faces)
        return (a * a + g * g) / (2 * len(X)), a * a, g * g

    mutants = [
        (check_quantize_nearest_level, _Mutant(quantize=quantize_floor)),
        (check_quantize_nearest_level, _Mutant(quantize=quantize_block_range)),
        (check_dequantize_error_bound, _Mutant(dequantize=dequantize_off_by_one)),
        (check_gl_hand_values, _Mutant(geometric_laplacian=gl_length_weights)),
        (check_gl_invariants, _Mutant(geometric_laplacian=gl_no_dedupe)),
        (check_nmsve_hand_values, _Mutant(nmsve=nmsve_squared)),
    ]
    for check, mut in mutants:
        with pytest.raises(AssertionError):
            check(O=mut)
