"""CPU checks of two pieces of arithmetic the GPU kernels rest on (no GPU).

1. The split-line LRMS sweeps of the split two-axis line kernel: a line of
   L labels (33 <= L <= 65) held as a first half of 32 labels and a second
   half of L - 32, each half swept on its own, then completed with one carry
   per direction (the backward sweep of the first half takes
   min(b, b[32] + lambda (32 - i)), the forward sweep of the second half
   min(f, f[31] + lambda (i - 31))), equals the sequential backward-then-
   forward sweeps of Sec. 3.2 (Eq. L_dec5, Eq. L_dec3) over the whole line,
   and both equal the truncated-linear distance transform by definition.

2. The shared-memory descriptors of the tensor-core convolutions: the halo
   image of a tile (halo row hy, channel chunk c of 8 channels, halo column
   hx at byte (hy * 4 + c) * 160 + hx * 16) read through the K-major
   descriptor of tap (dy, dx) (start dy * 640 + dx * 16 + pair * 320, LBO =
   160 along K, SBO = 640 along M) gives the im2col rows of the forward
   convolution, and read through the MN-major descriptors of the weight
   gradient (A: start dx * 16 + step * 1280, LBO = 640 along K, SBO = 160
   along M; B: the gradient tile at r * 512 + c * 128 + px * 16, LBO = 512,
   SBO = 128) gives the products of its definition.  The address rules are
   those of the no-swizzle canonical layouts (core matrices of 8 rows of
   16 bytes; LBO between core matrices along K, SBO along M or N)."""
import numpy as np
import pytest


def dt_definition(h, lam):
    """min over j of h[j] + lam |i - j| (the distance transform)."""
    L = len(h)
    idx = np.arange(L)
    return np.array([np.min(h + lam * np.abs(idx - i)) for i in range(L)])


def sweeps_sequential(h, lam):
    h = h.copy()
    for i in range(len(h) - 2, -1, -1):
        h[i] = min(h[i], h[i + 1] + lam)
    for i in range(1, len(h)):
        h[i] = min(h[i], h[i - 1] + lam)
    return h


def sweeps_split(h, lam):
    """Two halves of 32 and L - 32 labels, swept apart, completed by carries."""
    lo, hi = h[:32].copy(), h[32:].copy()
    for part in (lo, hi):  # backward sweeps of each half
        for i in range(len(part) - 2, -1, -1):
            part[i] = min(part[i], part[i + 1] + lam)
    cb = hi[0]  # b[32]
    lo = np.minimum(lo, cb + lam * (32 - np.arange(32)))
    for part in (lo, hi):  # forward sweeps of each half
        for i in range(1, len(part)):
            part[i] = min(part[i], part[i - 1] + lam)
    cf = lo[31]  # f[31]
    hi = np.minimum(hi, cf + lam * (np.arange(len(hi)) + 1))
    return np.concatenate([lo, hi])


@pytest.mark.parametrize("L", [33, 34, 47, 64, 65])
def test_split_sweeps_equal_sequential_sweeps(L):
    rng = np.random.default_rng(L)
    for trial in range(200):
        lam = int(rng.integers(0, 40))
        hi_val = int(rng.choice([3, 50, 10 ** 6]))
        h = rng.integers(0, hi_val, size=L).astype(np.int64)
        want = dt_definition(h, lam)
        assert np.array_equal(sweeps_sequential(h, lam), want)
        assert np.array_equal(sweeps_split(h, lam), want), (L, lam, trial)


def test_split_sweeps_catch_a_wrong_carry():
    """The identity test fails for a carry taken one label off."""
    rng = np.random.default_rng(1)
    h = rng.integers(0, 1000, size=65).astype(np.int64)
    h[40] = 0  # a strong source in the second half
    lo = h[:32].copy()
    for i in range(30, -1, -1):
        lo[i] = min(lo[i], lo[i + 1] + 5)
    hi = sweeps_sequential(h[32:], 5)
    wrong = np.minimum(lo, hi[0] + 5 * (31 - np.arange(32)))  # off by one label
    assert not np.array_equal(wrong, dt_definition(h, 5)[:32])


# --- tensor-core operand layouts -------------------------------------------

TX, TY = 8, 16                 # output tile
CHUNK, ROW = (TX + 2) * 16, 4 * (TX + 2) * 16   # 160, 640 bytes


def halo_image(halo):
    """halo [hy][hx][32 channels] (bf16 stand-in: int) -> byte-addressed image
    (a dict byte offset -> value, one entry per 2-byte element)."""
    img = {}
    HY, HX, _ = halo.shape
    for hy in range(HY):
        for hx in range(HX):
            for ch in range(32):
                c, e = divmod(ch, 8)
                img[(hy * 4 + c) * CHUNK + hx * 16 + e * 2] = halo[hy, hx, ch]
    return img


def read_kmajor(img, start, lbo, sbo, M, K):
    """A[m][k] of a K-major no-swizzle operand: core matrix (m // 8, k // 8)
    at start + (m // 8) sbo + (k // 8) lbo, row m % 8 at + 16 (m % 8),
    element k % 8 at + 2 (k % 8)."""
    return np.array([[img[start + (m // 8) * sbo + (k // 8) * lbo + (m % 8) * 16 + (k % 8) * 2]
                      for k in range(K)] for m in range(M)])


def read_mnmajor(img, start, lbo, sbo, M, K):
    """A[m][k] of an MN-major no-swizzle operand: core matrix (m // 8, k // 8)
    at start + (m // 8) sbo + (k // 8) lbo, row k % 8 at + 16 (k % 8),
    element m % 8 at + 2 (m % 8)."""
    return np.array([[img[start + (m // 8) * sbo + (k // 8) * lbo + (k % 8) * 16 + (m % 8) * 2]
                      for k in range(K)] for m in range(M)])


def test_forward_descriptors_give_im2col():
    rng = np.random.default_rng(3)
    halo = rng.integers(-500, 500, size=(TY + 2, TX + 2, 32))
    img = halo_image(halo)
    for dy in range(3):
        for dx in range(3):
            for pair in range(2):  # channels 16 pair .. 16 pair + 15: one MMA of K = 16
                A = read_kmajor(img, dy * ROW + dx * 16 + pair * 2 * CHUNK, CHUNK, ROW, 128, 16)
                # row m = output pixel (m % 8, m // 8) of the tile; k = channel 16 pair + k
                want = np.array([[halo[m // 8 + dy, m % 8 + dx, 16 * pair + k] for k in range(16)]
                                 for m in range(128)])
                assert np.array_equal(A, want), (dy, dx, pair)


def test_weight_gradient_descriptors_give_the_products():
    rng = np.random.default_rng(4)
    halo = rng.integers(-500, 500, size=(TY + 3, TX + 2, 32))  # 19 rows: dy = 0..3
    img = halo_image(halo)
    gt = rng.integers(-500, 500, size=(TY, TX, 32))
    gimg = {}
    for r in range(TY):
        for px in range(TX):
            for co in range(32):
                c, e = divmod(co, 8)
                gimg[r * 512 + c * 128 + px * 16 + e * 2] = gt[r, px, co]
    for dx in range(3):
        D = np.zeros((128, 32), np.int64)
        for step in range(TY // 2):  # 16 pixels (two tile rows) per MMA
            A = read_mnmajor(img, dx * 16 + step * 2 * ROW, ROW, CHUNK, 128, 16)
            B = read_mnmajor(gimg, step * 1024, 512, 128, 32, 16)  # B[n = co][k = pixel]
            D += A.astype(np.int64) @ B.T.astype(np.int64)
        # row m = (dy, ci) = 32 dy + ci: sum over the tile's pixels of x[p + (dy, dx)][ci] g[p][co]
        for dy in range(3):
            want = np.einsum("rpc,rpo->co", halo[dy:dy + TY, dx:dx + TX, :].astype(np.int64),
                             gt.astype(np.int64))
            assert np.array_equal(D[32 * dy:32 * dy + 32], want), (dx, dy)
