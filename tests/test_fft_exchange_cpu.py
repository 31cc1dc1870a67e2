"""Shared-memory addressing of the FFT exchanges, restated on the CPU.

The register FFT of csrc/hd_fft.cuh runs radix-E passes on E values per
thread and exchanges values between passes through a padded shared-memory
buffer of FftShape<S, E>::SMEM slots per transform.  This file restates the
addresses that fft_exchange computes (writes after pass k, reads before pass
k + 1; the inverse uses the same addresses with the directions swapped) for
every (S, E) the library compiles, and checks:

* every access stays inside the buffer (index < SMEM), and the writes and the
  reads of one exchange each touch every logical slot exactly once;
* the shortcut form of a padded index (one padded base per group of accesses)
  equals the padded index itself;
* for E = 8 and E = 16 with 32 or more threads per transform, every 64-bit
  access of a half-warp (16 lanes x 8 bytes, FP32 complex) hits 16 distinct
  bank pairs: the exchanges are free of bank conflicts;
* the Hermitian split's mirror reads stay inside the buffer.
"""
import math

import pytest

F32 = [(2, 2), (4, 4), (8, 8), (16, 8), (32, 8), (64, 8), (128, 8), (256, 8), (512, 8), (1024, 8), (2048, 8),
       (4096, 8), (512, 4), (1024, 4), (2048, 4), (256, 16), (512, 16), (1024, 16), (2048, 16), (4096, 16)]
COLS = [(S, 8 if S <= 128 else 16) for S in (8, 16, 32, 64, 128, 256, 512, 1024, 2048, 4096)]


class Shape:
    def __init__(self, S, E):
        self.S, self.E, self.T = S, E, S // E
        LS, LE = int(math.log2(S)), int(math.log2(E))
        self.KFULL = LS // LE
        self.K = self.KFULL + (1 if LS % LE else 0)
        self.last = 1 << (LS % LE)
        self.SMEM = S + (S // 8 if E == 8 else S // 16)

    def radix(self, k):
        return self.E if k < self.KFULL else self.last

    def sub(self, k):
        n = self.S
        for j in range(k):
            n //= self.radix(j)
        return n


def exchange(sh, k, cst=1, one_pad=False):
    """(writes, reads) of exchange k: per warp-wide access, the list of
    (logical slot, padded index) over the T threads of one transform.
    one_pad: one pad element per 16 everywhere (the layout without the second
    pad element of the radix-8 reads)."""
    R, Rn = sh.radix(k), sh.radix(k + 1)
    V = sh.S // R
    Qn = sh.sub(k + 1) // Rn
    padm = 2 if (cst == 1 and Rn == 8 and 1 < Qn < 16 and not one_pad) else 1

    def padk(a):
        return a + (a >> 4) * padm

    writes, reads = [], []
    for beta in range(sh.E // R):
        for k1 in range(R):
            acc = []
            for tau in range(sh.T):
                nu = tau + sh.T * beta
                logical = nu + V * k1
                idx = padk(nu) + V * k1 + (V // 16) * padm * k1 if V % 16 == 0 else padk(logical)
                acc.append((logical, idx, padk(logical)))
            writes.append(acc)
    for beta in range(sh.E // Rn):
        for i in range(Rn):
            acc = []
            for tau in range(sh.T):
                nu = tau + sh.T * beta
                b, c = nu // Qn, nu & (Qn - 1)
                base = b * Rn * Qn + c
                logical = base + i * Qn
                idx = padk(base) + i * Qn + (Qn // 16) * padm * i if Qn % 16 == 0 else padk(logical)
                acc.append((logical, idx, padk(logical)))
            reads.append(acc)
    return writes, reads


def conflict_degree(idxs):
    """Largest number of distinct 8-byte words of one half-warp in one bank pair."""
    worst = 1
    for w0 in range(0, len(idxs), 32):
        warp = idxs[w0:w0 + 32]
        for h in range(0, len(warp), 16):
            banks = {}
            for a in warp[h:h + 16]:
                banks.setdefault(a % 16, set()).add(a)
            worst = max(worst, max(len(v) for v in banks.values()))
    return worst


@pytest.mark.parametrize("S,E", F32)
def test_exchange_in_bounds_and_bijective(S, E):
    sh = Shape(S, E)
    for k in range(sh.K - 1):
        for accs in exchange(sh, k):
            logical = sorted(l for acc in accs for l, _, _ in acc)
            assert logical == list(range(S)), (S, E, k)
            for acc in accs:
                for l, idx, full in acc:
                    assert idx == full, (S, E, k, l)          # shortcut form == padded index
                    assert 0 <= idx < sh.SMEM, (S, E, k, l, idx)
            padded = [idx for acc in accs for _, idx, _ in acc]
            assert len(set(padded)) == S


@pytest.mark.parametrize("S,E", [(S, E) for S, E in F32 if E in (8, 16) and S // E >= 32])
def test_exchange_conflict_free(S, E):
    sh = Shape(S, E)
    for k in range(sh.K - 1):
        writes, reads = exchange(sh, k)
        for acc in writes + reads:
            assert conflict_degree([idx for _, idx, _ in acc]) == 1, (S, E, k)


@pytest.mark.parametrize("S,E", COLS)
def test_column_exchanges_in_bounds(S, E):
    """Column tiles interleave CST transforms (one pad element per 16): every
    slot of every transform stays inside its interleaved buffer."""
    sh = Shape(S, E)
    for k in range(sh.K - 1):
        for accs in exchange(sh, k, cst=4):
            for acc in accs:
                for l, idx, full in acc:
                    assert idx == full and 0 <= idx < sh.SMEM


@pytest.mark.parametrize("S,E", F32)
def test_hermitian_split_reads_in_bounds(S, E):
    """The split of two Hermitian inverses stores slot j at padidx(j) and reads
    padidx((S - j) mod S) (one pad element per 16), within SMEM."""
    sh = Shape(S, E)
    for j in range(S):
        for x in (j, (S - j) & (S - 1)):
            assert x + (x >> 4) < sh.SMEM


def test_single_pad_has_the_conflicts_the_second_pad_removes():
    """Without the second pad element, the radix-8 reads with 1 < Q < 16 meet
    two words in one bank pair: the model sees the conflicts the layout
    avoids."""
    found = []
    for S, E in [(S, 8) for S in (256, 512, 1024, 2048, 4096)]:
        sh = Shape(S, E)
        for k in range(sh.K - 1):
            _, reads = exchange(sh, k, one_pad=True)
            d = max(conflict_degree([idx for _, idx, _ in acc]) for acc in reads)
            if d > 1:
                found.append((S, k, d))
    assert found and all(d == 2 for _, _, d in found), found
