"""The byte-SIMD site rules of the CUDA passes, transcribed here in numpy and
checked on the CPU against brute force and the oracle (no GPU needed).

These are the arithmetic identities the kernels rely on, stated once more in
plain array code so that a mistake in the identity (not only in its CUDA
spelling) fails without a GPU:

- Metropolis (pass_u8.cuh, delta_index): for spins below 2^QB the per-byte
  sums X = 16 #[P != n] and Y = 16 #[S != n] over the four neighbours give
  16 (4 + dE) = 64 + X - Y, and the black pass's unequal count after the
  update is X where accepted, Y elsewhere; for wider spins the zero-byte
  test gives the same counts.
- Heat bath (heatbath.cuh, hb_word with the 64-entry pattern table): the new
  spins of four sites at once equal the oracle's one-site rule (Sec. 6's
  heat bath under the reading documented with the oracle).

The GPU parity tests compare the kernels themselves with the oracle; these
tests pin the word-level reasoning behind them.
"""
import numpy as np
import pytest

import oracle

M32 = 0xFFFFFFFF


def _words(b):
    """bytes (..., 4) -> uint64 words holding 32-bit values"""
    b = b.astype(np.uint64)
    return b[..., 0] | (b[..., 1] << 8) | (b[..., 2] << 16) | (b[..., 3] << 24)


def _byte(w, k):
    return (w >> np.uint64(8 * k)) & np.uint64(0xFF)


# ------------------------------------------------------------ Metropolis

def _ne16_sum4(QB, xs):
    """16 * [byte != 0] per byte summed over four words (spins < 2^QB)."""
    u = np.uint64
    if QB == 4:
        K, M = u(0x0F0F0F0F), u(0x10101010)
        return sum(((x + K) & M) for x in xs)
    if QB == 5:
        K, M = u(0x1F1F1F1F), u(0x20202020)
        return sum(((x + K) & M) for x in xs) >> u(1)
    if QB == 6:
        K, M = u(0x3F3F3F3F), u(0x40404040)
        return ((((xs[0] + K) & M) + ((xs[1] + K) & M)) >> u(2)) + \
            ((((xs[2] + K) & M) + ((xs[3] + K) & M)) >> u(2))
    if QB == 7:
        K, M = u(0x7F7F7F7F), u(0x80808080)
        return sum((((x + K) & M) >> u(3)) for x in xs)
    K, M = u(0x7F7F7F7F), u(0x80808080)
    return sum((((((x & K) + K) | x) & M) >> u(3)) for x in xs)


def _delta_index(QB, S, P, U, D, C, W):
    """(idx, no16, nn16) per word, as delta_index computes them."""
    u = np.uint64
    if QB <= 5:
        K = u(0x01010101 * ((1 << QB) - 1))
        M = u(0x01010101 * (1 << QB))
        a = [((S ^ N) + K) & u(M32) for N in (U, D, C, W)]
        b = [((P ^ N) + K) & u(M32) for N in (U, D, C, W)]
        X = sum(x & M for x in b)
        Y = sum(y & M for y in a)
        if QB == 5:
            X >>= u(1)
            Y >>= u(1)
        return ((X + u(0x40404040)) - Y) & u(M32), Y, X
    no = _ne16_sum4(QB, [S ^ N for N in (U, D, C, W)])
    nn = _ne16_sum4(QB, [P ^ N for N in (U, D, C, W)])
    return (u(0x40404040) + nn - no) & u(M32), no, nn


@pytest.mark.parametrize("QB", [4, 5, 6, 7, 8])
def test_metropolis_decision_index_and_counts(QB):
    rng = np.random.default_rng(100 + QB)
    n = 40000
    # few distinct values so that equal neighbours are common
    vals = rng.integers(0, 1 << QB, size=(n, 1, 3))
    pick = rng.integers(0, 3, size=(n, 6, 4))
    b = np.take_along_axis(np.broadcast_to(vals, (n, 6, 3)), pick, axis=2)
    b[: n // 4] = rng.integers(0, 1 << QB, size=(n // 4, 6, 4))
    S, P, U, D, C, W = (_words(b[:, i]) for i in range(6))
    idx, no16, nn16 = _delta_index(QB, S, P, U, D, C, W)
    acc = rng.integers(0, 2, size=(n, 4))
    m = _words(acc * 0xFF)
    nf16 = (nn16 & m) | (no16 & (m ^ np.uint64(M32)))
    for k in range(4):
        s, p = b[:, 0, k], b[:, 1, k]
        nb = b[:, 2:, k]
        n_old = (nb == s[:, None]).sum(1)
        n_new = (nb == p[:, None]).sum(1)
        assert np.array_equal(_byte(idx, k), 16 * (4 + n_old - n_new))
        assert np.array_equal(_byte(no16, k), 16 * (4 - n_old))
        assert np.array_equal(_byte(nn16, k), 16 * (4 - n_new))
        final_unequal = np.where(acc[:, k] == 1, 4 - n_new, 4 - n_old)
        assert np.array_equal(_byte(nf16, k), 16 * final_unequal)


# -------------------------------------------------------------- heat bath

def _pattern_table(W, q, m):
    """hb_pattern_entry for the 64 codes: rows (s1, s2, s3, s4, Z), the
    cumulative excesses W[c] - W[0] of the neighbours' classes (a repeated
    neighbour adds none) and Z = s4 + q 2^m."""
    ex = [0] + [int(W[c]) - int(W[0]) for c in range(1, 5)] + [0]
    t = np.zeros((64, 5), dtype=np.uint64)
    for code in range(64):
        e01, e02, e03, e12, e13, e23 = ((code >> i) & 1 for i in range(6))
        f1, f2, f3 = e01 ^ 1, (e02 | e12) ^ 1, (e03 | e13 | e23) ^ 1
        c = [1 + e01 + e02 + e03, 1 + e12 + e13 if f1 else 5,
             1 + e23 if f2 else 5, 1 if f3 else 5]
        s = np.cumsum([ex[x] for x in c]) & M32
        t[code, :4] = s
        t[code, 4] = (int(s[3]) + ((q << m) & M32)) & M32
    return t


def _hb_word(QB, U, D, Lw, Rw, uw, tab, m):
    """hb_word: new spins (word) of four sites from their neighbour words
    and Philox words uw (n, 4)."""
    u = np.uint64

    def eq_at(a, b, t):
        """[a == b] per byte at bit t: straight from bit t of x + 2^t - 1
        when t >= QB, else from bit QB moved down."""
        p = max(t, QB)
        K, M = u(0x01010101 * ((1 << p) - 1)), u(0x01010101 * (1 << p))
        e = ((((a ^ b) + K) & u(M32)) ^ u(M32)) & M
        return e >> u(p - t)

    # four times the pattern code per byte: the equalities at bits 2..7
    CODE = eq_at(U, D, 2) | eq_at(U, Lw, 3) | eq_at(U, Rw, 4) | \
        eq_at(D, Lw, 5) | eq_at(D, Rw, 6) | eq_at(Lw, Rw, 7)
    assert not (CODE & u(0x03030303)).any()
    N = np.zeros((U.size, 4), dtype=np.uint64)
    for b in range(4):
        e = tab[(_byte(CODE, b) >> u(2)).astype(np.int64)]
        r = (uw[:, b].astype(np.uint64) * e[:, 4]) >> u(32)
        n = (((r - e[:, 3]) & u(M32)) >> u(m)) & u(0xFF)
        # later (lower) bounds overwrite: the first interval holding r wins
        for i, src in ((3, Rw), (2, Lw), (1, D), (0, U)):
            n = np.where(r < e[:, i], _byte(src, b), n)
        N[:, b] = n
    return _words(N)


@pytest.mark.parametrize("q,beta,nv", [(3, 0.8, 3), (9, np.log(4.0), 9),
                                       (9, 1.1, 3), (16, 1.3, 16),
                                       (24, 1.2, 24), (24, 1.2, 3),
                                       (40, 3.0, 4), (64, 2.0, 64),
                                       (64, 0.0, 64), (5, 5.5, 5)])
def test_heatbath_word_rule_equals_oracle(q, beta, nv):
    QB = 4 if q <= 16 else (5 if q <= 32 else 6)
    L, seed, t = 32, 17 + q, 3
    W, m = oracle.heatbath_weights(beta, q)
    tab = _pattern_table(W, q, m)
    rng = np.random.default_rng(q * 7 + nv)
    pre = rng.integers(0, nv, size=(L, L), dtype=np.uint8)
    ii, jj = np.nonzero((np.add.outer(np.arange(L), np.arange(L)) % 2) == 0)
    idx = (ii * L + jj).astype(np.int64)
    expect = oracle.sweep_sites(pre, q, seed, t, beta, idx,
                                update=oracle.HEATBATH)
    # four consecutive white sites of a row form one word, as in the kernel
    nb = np.stack([pre[(ii - 1) % L, jj], pre[(ii + 1) % L, jj],
                   pre[ii, (jj - 1) % L], pre[ii, (jj + 1) % L]], axis=1)
    nb = nb.reshape(-1, 4, 4)                     # (words, site, neighbour)
    U, D, Lw, Rw = (_words(nb[:, :, j]) for j in range(4))
    uw = np.array([oracle.site_word(seed, t, 0, int(k) >> 1) for k in idx],
                  dtype=np.uint64).reshape(-1, 4)
    N = _hb_word(QB, U, D, Lw, Rw, uw, tab, m)
    got = np.stack([_byte(N, b) for b in range(4)], axis=1).reshape(-1)
    assert np.array_equal(got.astype(np.uint8), expect)
