"""The arithmetic of the one-router streaming kernels, restated on the host and checked against the
definitions it stands for, exhaustively over the 16-bit values (the kernels themselves are checked
against the oracle by the GPU tests; this pins the reasoning they are built on):

- a recorder's distance is 65535 for the stamp 0xFFFF, else (tm - x) mod 65535 (Sec. 3.2 recorders
  kept as stamps beside a clock tm in 0..65534);
- inside the window (distance < k) is: x unchanged by clamping into [lo, hi] (one range), or into
  [lo, 65534] or [0, tm] when the window wraps past 65534 (tm + 1 < k);
- a vector holds the stamp xe exactly when some half of x ^ xe is zero (min over halves, then
  min with 1, tested against 0x00010001);
- the touch byte of vector it*32 + lane of an estimator is stored at lane * (eta / 256) + it: a
  bijection on the estimator's bytes that makes each lane's bytes contiguous."""
import numpy as np

X = np.arange(65536, dtype=np.int64)       # every 16-bit recorder value


def distance(x, tm):
    return np.where(x == 0xFFFF, 65535, (tm - x) % 65535)


def clock(tm, k):
    """lo, hi, wrap of the window as the kernels' clock sets them."""
    wrap = tm + 1 < k
    lo = tm + 65536 - k if wrap else tm + 1 - k
    hi = 65534 if wrap else tm
    return lo, hi, wrap


def clamp_inside(x, lo, hi):
    return np.maximum(np.minimum(x, hi), lo) == x


def window(x, tm, k):
    lo, hi, wrap = clock(tm, k)
    inside = clamp_inside(x, lo, hi)
    if wrap:
        inside |= clamp_inside(x, 0, tm)
    return inside


def test_clamp_window_is_distance_below_k_for_every_stamp():
    ks = (1, 2, 3, 60, 300, 4096, 65533, 65534)
    for k in ks:
        tms = {0, 1, 2, k - 2, k - 1, k, 65533, 65534, 30000, 12345}
        for tm in sorted(t for t in tms if 0 <= t <= 65534):
            got = window(X, tm, k)
            want = distance(X, tm) < k
            assert np.array_equal(got, want), (k, tm, np.flatnonzero(got != want)[:5])


def test_window_of_distances_is_one_range():
    # the allocation-free regain reads distances: lo = 0, hi = k - 1, never wrapping
    for k in (1, 60, 65534):
        assert np.array_equal(clamp_inside(X, 0, k - 1), X < k)


def test_expiring_stamp_lies_outside_the_window():
    # xe = tm + 1 mod 65535 is the stamp whose distance reaches 65535 at the advance; the window
    # count taken before the expiry must not include it
    for k in (1, 60, 65534):
        for tm in (0, 1, k - 2, k - 1, 65533, 65534):
            if not 0 <= tm <= 65534:
                continue
            xe = 0 if tm + 1 >= 65535 else tm + 1
            assert not window(np.array([xe]), tm, k)[0]
            assert distance(np.array([xe]), tm)[0] == 65534


def umin2(a, b):
    lo = np.minimum(a & 0xFFFF, b & 0xFFFF)
    hi = np.minimum(a >> 16, b >> 16)
    return (hi << 16) | lo


def any_eq8(words, xe):
    xe2 = xe | (xe << 16)
    m = umin2(umin2(words[0] ^ xe2, words[1] ^ xe2), umin2(words[2] ^ xe2, words[3] ^ xe2))
    return umin2(m, 0x00010001) != 0x00010001


def test_vector_equality_test_is_exact():
    rng = np.random.default_rng(5)
    n = 200_000
    for xe in (0, 1, 1000, 65534):
        halves = rng.integers(0, 65536, size=(n, 8), dtype=np.int64)
        plant = rng.random(n) < 0.3
        halves[plant, rng.integers(0, 8, size=int(plant.sum()))] = xe
        words = [(halves[:, 2 * i + 1] << 16) | halves[:, 2 * i] for i in range(4)]
        assert np.array_equal(any_eq8(words, xe), (halves == xe).any(axis=1))


def touch_pos(log2_eta, x):
    if log2_eta < 8:
        return x
    vi = x >> 3
    return ((((vi & 31) << (log2_eta - 8)) | (vi >> 5)) << 3) | (x & 7)


def test_touch_positions_are_a_bijection_with_contiguous_lane_bytes():
    for log2_eta in range(5, 16):
        eta = 1 << log2_eta
        x = np.arange(eta, dtype=np.int64)
        pos = touch_pos(log2_eta, x)
        assert np.array_equal(np.sort(pos), x)                  # a permutation of the eta bits
        assert np.array_equal(pos & 7, x & 7)                   # a recorder keeps its bit in the byte
        if log2_eta < 8:
            continue
        iters = eta >> 8
        vi = x >> 3
        lane, it = vi & 31, vi >> 5
        byte = pos >> 3
        assert np.array_equal(byte, lane * iters + it)
        # the bytes of one lane's group of min(8, iters) vectors are contiguous and aligned
        m = min(8, iters)
        for ln in (0, 7, 31):
            for it0 in range(0, iters, 8):
                sel = (lane == ln) & (it >= it0) & (it < it0 + m)
                got = np.unique(byte[sel])
                assert got[0] % m == 0 and np.array_equal(got, np.arange(got[0], got[0] + m))
