"""Host-side checks of the shared-memory FFT schemes of the CUDA kernels (no GPU).

The kernels' index arithmetic is restated here in Python:
* the radix-8 Stockham stages (stockham.cuh: stage_r8, the leading radix-2/4
  stage, the stage-grouped twiddle table of api.cu::staged_twiddles8) and the
  4 x 8 x 8 x 4 plan of the ny = 1024 column kernel (api.cu::cols1024_twiddles)
  reproduce numpy's FFT;
* the radix-8 buffer paddings j + c (j >> 4) keep every stage's reads and writes
  free of shared-memory bank conflicts;
* the XOR swizzle of the Bluestein work buffer (fft_smem.cuh::blu_swz) keeps the
  bit-reversed and strided accesses of the in-place transform at <= 2 distinct
  elements per bank and half-warp.
Banks: 32 four-byte banks; a 64-bit access is served 16 lanes at a time.
"""
import numpy as np
import pytest


def bitrev(x, lg):
    return int(format(x, f"0{lg}b")[::-1], 2) if lg else 0


def multiplicity(addrs, words=2):
    """Distinct elements hitting the busiest bank in one 16-lane phase."""
    banks = {}
    for a in addrs:
        for w in range(words * a, words * a + words):
            banks.setdefault(w % 32, set()).add(a)
    return max(len(v) for v in banks.values())


# --- radix-8 Stockham ------------------------------------------------------------

def twiddles8(n):
    lg = n.bit_length() - 1
    p0 = 1 << (lg % 3)
    t = np.zeros(n, complex)
    p = p0
    while 8 * p <= n:
        for q in range(1, 8):
            for k in range(p):
                t[(p - p0) + (q - 1) * p + k] = np.exp(-2j * np.pi * q * k * (n // (8 * p)) / n)
        p *= 8
    return t, p0


def dft(v, inv):
    return np.fft.ifft(v) * len(v) if inv else np.fft.fft(v)


def stockham8(x, inv=False):
    n = len(x)
    lg = n.bit_length() - 1
    r0 = lg % 3
    tw, p0 = twiddles8(n)
    a = np.asarray(x, complex).copy()
    if r0:
        r = 1 << r0
        q = n // r
        b = np.zeros(n, complex)
        for i in range(q):
            b[r * i:r * i + r] = dft(np.array([a[i + m * q] for m in range(r)]), inv)
        a = b
    p = p0 if r0 else 1
    while p < n:
        q = n // 8
        b = np.zeros(n, complex)
        for i in range(q):
            k = i & (p - 1)
            v = np.array([a[i + m * q] for m in range(8)])
            if p > 1:
                for m in range(1, 8):
                    w = tw[(p - p0) + (m - 1) * p + k]
                    v[m] *= np.conj(w) if inv else w
            y = dft(v, inv)
            j = ((i - k) << 3) + k
            for r in range(8):
                b[j + r * p] = y[r]
        a = b
        p *= 8
    return a


@pytest.mark.parametrize("n", [128, 256, 512, 1024])
@pytest.mark.parametrize("inv", [False, True])
def test_radix8_stockham_is_the_dft(n, inv):
    rng = np.random.default_rng(n)
    x = rng.standard_normal(n) + 1j * rng.standard_normal(n)
    ref = np.fft.ifft(x) * n if inv else np.fft.fft(x)
    assert np.abs(stockham8(x, inv) - ref).max() <= 1e-12 * n


def test_cols1024_plan_is_the_dft():
    n = 1024
    tw = np.zeros(n, complex)
    for p in (4, 32):
        for q in range(1, 8):
            for k in range(p):
                tw[(p - 4) + (q - 1) * p + k] = np.exp(-2j * np.pi * q * k * (n // (8 * p)) / n)
    for q in range(1, 4):
        for k in range(256):
            tw[252 + (q - 1) * 256 + k] = np.exp(-2j * np.pi * q * k / n)
    rng = np.random.default_rng(7)
    x = rng.standard_normal(n) + 1j * rng.standard_normal(n)
    for inv in (False, True):
        c = np.conj if inv else (lambda w: w)
        a = np.zeros(n, complex)
        for t in range(256):                       # radix 4, span 1, in registers
            a[4 * t:4 * t + 4] = dft(np.array([x[t + 256 * r] for r in range(4)]), inv)
        for p in (4, 32):                           # radix 8, spans 4 and 32
            b = np.zeros(n, complex)
            for i in range(128):
                k = i & (p - 1)
                v = np.array([a[i + m * 128] for m in range(8)])
                for m in range(1, 8):
                    v[m] *= c(tw[(p - 4) + (m - 1) * p + k])
                y = dft(v, inv)
                for r in range(8):
                    b[((i - k) << 3) + k + r * p] = y[r]
            a = b
        out = np.zeros(n, complex)
        for t in range(256):                       # radix 4, span 256, in registers
            v = np.array([a[t + 256 * r] * (c(tw[252 + (r - 1) * 256 + t]) if r else 1) for r in range(4)])
            y = dft(v, inv)
            for q in range(4):
                out[t + 256 * q] = y[q]
        ref = np.fft.ifft(x) * n if inv else np.fft.fft(x)
        assert np.abs(out - ref).max() <= 1e-12 * n


def padc(j, c):
    return j + c * (j >> 4)


@pytest.mark.parametrize("n", [128, 256, 512, 1024])
def test_radix8_paddings_are_conflict_free(n):
    lg = n.bit_length() - 1
    r0 = lg % 3
    spans, p = [], (1 << r0) if r0 else 1
    while p < n:
        spans.append(p)
        p *= 8
    worst = 1
    if r0:                                          # leading stage: reads c = 0, writes c = 1
        r = 1 << r0
        q = n // r
        for m in range(r):
            for base in range(0, q, 16):
                lanes = range(base, base + 16)
                worst = max(worst, multiplicity([i + m * q for i in lanes]),
                            multiplicity([padc(r * i + m, 1) for i in lanes]))
    for si, p in enumerate(spans):
        cout = 0 if si == len(spans) - 1 else (1 if p == 1 else 2)
        cin = 0 if (si == 0 and not r0) else (1 if si == 0 else (1 if spans[si - 1] == 1 else 2))
        q = n // 8
        for r in range(8):
            for base in range(0, q, 16):
                lanes = range(base, min(base + 16, q))
                wr = [padc(((i - (i & (p - 1))) << 3) + (i & (p - 1)) + r * p, cout) for i in lanes]
                rd = [padc(i + r * q, cin) for i in lanes]
                worst = max(worst, multiplicity(wr), multiplicity(rd))
    assert worst == 1


# --- Bluestein work buffer --------------------------------------------------------

def blu_swz(p, lg):
    return p ^ (((p >> 4) ^ (p >> (lg - 4))) & 15)


def bluestein_patterns(lg, n_points):
    """Per warp instruction: the 32 element indices of the in-place transform's
    accesses (input scatter, stages in threes / a pair / a single, the
    bit-reversed pointwise pass, the natural-order output)."""
    L = 1 << lg
    pats = [[bitrev(x, lg) for x in range(x0, x0 + 32)] for x0 in range(0, L, 32)]
    s = 0
    while s + 2 < lg:
        hs = 1 << s
        for g0 in range(0, L >> 3, 32):
            for j in range(8):
                pats.append([((g >> s) << (s + 3)) + (g & (hs - 1)) + j * hs for g in range(g0, g0 + 32)])
        s += 3
    if s + 1 < lg:
        hs = 1 << s
        for g0 in range(0, L >> 2, 32):
            for j in range(4):
                pats.append([((g >> s) << (s + 2)) + (g & (hs - 1)) + j * hs for g in range(g0, g0 + 32)])
        s += 2
    if s < lg:
        hs = 1 << s
        for k0 in range(0, L >> 1, 32):
            for j in range(2):
                pats.append([((k >> s) << (s + 1)) + (k & (hs - 1)) + j * hs for k in range(k0, k0 + 32)])
    for i0 in range(0, L, 32):
        act = [i for i in range(i0, i0 + 32) if i <= bitrev(i, lg)]
        pats.append(act)
        pats.append([bitrev(i, lg) for i in act])
    half = n_points // 2 + 1
    pats += [list(range(k0, min(k0 + 32, half))) for k0 in range(0, half, 32)]
    pats += [[(n_points - k) if k else 0 for k in range(k0, min(k0 + 32, half))] for k0 in range(0, half, 32)]
    return pats


@pytest.mark.parametrize("lg,n_points", [(9, 200), (10, 500), (11, 1000), (12, 2000), (13, 4000)])
def test_bluestein_swizzle(lg, n_points):
    L = 1 << lg
    assert sorted(blu_swz(p, lg) for p in range(L)) == list(range(L))     # a permutation of the buffer
    plain = swz = 0
    for ins in bluestein_patterns(lg, n_points):
        for half in (ins[:16], ins[16:]):
            if half:
                plain = max(plain, multiplicity(half))
                swz = max(swz, multiplicity([blu_swz(p, lg) for p in half]))
    assert swz <= 2
    assert plain >= 8                                                      # what the swizzle removes


# --- rows-C (nx = 1024) TMA stage buffer ------------------------------------------

RC_BOX, M, FH = 176, 512, 4


def wavefronts(byte_addrs, width=16):
    """Shared-memory wavefronts of one 128-bit warp access: served a quarter warp (8
    lanes) at a time; a phase takes as many wavefronts as the busiest of the 32 four-byte
    banks has distinct words."""
    n = 0
    for q in range(4):
        banks = {}
        for a in byte_addrs[8 * q:8 * q + 8]:
            for w in range(a // 4, (a + width) // 4):
                banks.setdefault(w % 32, set()).add(w)
        n += max(len(v) for v in banks.values())
    return n


def test_rows_c_stage_halves():
    """The six TMA boxes of a rows-C stage (2 complex x 176 kx rows each: rows y0, y0+1
    into half 0, rows y0+2, y0+3 into half 1) start on 128-byte boundaries, their x
    coordinates (floats) are 16-byte multiples, they tile each half's [kx][2] rows 0..527
    with no overlap, and the split's reads of kx = t, M - t, t + 256, 256 - t from both
    halves take 4 wavefronts per warp access (the single [kx][4] array took 8)."""
    rows = 3 * RC_BOX
    assert rows >= M + 1
    cover = {}
    for hf in range(2):
        for buf in range(2):
            for b in range(3):
                start = ((2 * hf + buf) * rows + b * RC_BOX) * 2 * 8      # bytes: float2 index * 8
                assert start % 128 == 0 and (RC_BOX * 16) % 128 == 0
                for yb in (0, 1, 255):
                    x = 2 * FH * yb + 4 * hf
                    assert (x * 4) % 16 == 0
                for r in range(RC_BOX):
                    key = (hf, buf, b * RC_BOX + r)
                    assert key not in cover
                    cover[key] = start + 16 * r
    assert len(cover) == 2 * 2 * rows
    assert max(cover.values()) + 16 <= 2 * rows * FH * 8            # inside the staging area
    for w in range(8):
        lanes = [32 * w + j for j in range(32)]
        for kx in (lambda t: t, lambda t: M - t, lambda t: t + 256, lambda t: 256 - t):
            for hf in range(2):
                addrs = [((2 * hf) * rows + kx(t)) * 16 for t in lanes]
                assert all(0 <= kx(t) <= M for t in lanes)
                assert wavefronts(addrs) == 4
            old = [kx(t) * 32 for t in lanes]                        # [kx][4]: 32 bytes per lane
            assert wavefronts(old) == 8 and wavefronts([a + 16 for a in old]) == 8
