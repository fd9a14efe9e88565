"""The index identities the line-pass kernels rely on, checked exhaustively on the CPU for every FFT
plan and tile geometry the passes launch (restated here from the kernels' definitions):

- padded shared-memory offsets (fft_fixed.cuh, pad_step): with fft_pad(i) = i + i/16, a Stockham stage
  of radix RAD on sub-transforms of length NS reads j + r NB (NB = L/RAD) and writes base + r NS
  (base = (j - k) RAD + k, k = j mod NS); for every such access fft_pad(first + d) = fft_pad(first) +
  d + d/16, so the r-th operand is a constant offset from the first;
- stepped tile indexing (passes.cuh, TileWalk): visiting the elements e = tid, tid + nthr, ... < B n of
  a tile by stepping (line, position, global index) gives exactly the per-element formulas.
"""
import pytest


def fft_pad(i):
    return i + (i >> 4)


def pad_step(d):
    return d + (d >> 4)


@pytest.mark.parametrize("logr", [2, 3, 4])
def test_padded_offsets_are_constant_steps(logr):
    for log2L in range(2, 13):
        L = 1 << log2L
        nfull = log2L // logr
        loglast = log2L - nfull * logr
        NS = 1
        for s in range(nfull + (1 if loglast else 0)):
            RAD = 1 << (logr if s < nfull else loglast)
            NB = L // RAD
            for j in range(NB):
                k = j & (NS - 1)
                base = (j - k) * RAD + k
                for r in range(RAD):
                    assert fft_pad(j + r * NB) == fft_pad(j) + pad_step(r * NB), (logr, log2L, s, j, r)
                    assert fft_pad(base + r * NS) == fft_pad(base) + pad_step(r * NS), (logr, log2L, s, j, r)
            NS *= RAD


def _per_element(xax, B, log2B, n, nthr, tid, line0, hi, lo0, stride, nlines):
    out, e = [], tid
    while e < B * n:
        if xax:
            l, pos = (0, e) if B == 1 else (e // n, e - (e // n) * n)
            out.append((l, pos, (line0 + l) * n + pos, line0 + l < nlines))
        else:
            pos, l = e >> log2B, e & (B - 1)
            out.append((l, pos, lo0 + l + pos * stride + hi * stride * n, lo0 + l < stride))
        e += nthr
    return out


def _stepped(xax, B, log2B, n, nthr, tid, line0, hi, lo0, stride, nlines):
    out = []
    if xax:
        l = 0 if B == 1 else tid // n
        pos, g, dg, dpos, valid = tid - l * n, line0 * n + tid, nthr, nthr, line0 + l < nlines
    else:
        l, pos, dpos = tid & (B - 1), tid >> log2B, nthr >> log2B
        g, dg, valid = lo0 + l + pos * stride + hi * stride * n, dpos * stride, lo0 + l < stride
    while (pos < n and l < B) if xax else pos < n:
        out.append((l, pos, g, valid))
        pos += dpos
        g += dg
        if xax and B > 1:
            while pos >= n:
                pos -= n
                l += 1
            valid = line0 + l < nlines
    return out


@pytest.mark.parametrize("n", [3, 7, 31, 127, 255, 511, 1023, 2047])
def test_stepped_tile_indexing_matches_the_formulas(n):
    L = 2 * (n + 1)
    nl = n * n
    for nt in {max(1, L // 8), max(1, L // 4)}:
        for B in (1, 2, 4, 8, 16):
            nthr = B * nt
            if nthr > 512:
                continue
            log2B = B.bit_length() - 1
            for xax in (True, False):
                if xax:
                    geos = [(t * B, 0, 0, 1) for t in (0, (nl + B - 1) // B - 1)]
                else:
                    ti = (n + B - 1) // B
                    geos = [(0, h, t * B, n) for h in (0, n - 1) for t in (0, ti - 1)]
                for line0, hi, lo0, stride in geos:
                    for tid in sorted({0, 1, nt - 1, nthr // 2, nthr - 1}):
                        args = (xax, B, log2B, n, nthr, tid, line0, hi, lo0, stride, nl)
                        assert _stepped(*args) == _per_element(*args), args
