"""Index design of the register-resident binary32 Jacobi start (N = 32):
the pair order and the skewed register layout it relies on, checked on the
host.  No GPU.

Round r pairs every index i with i ^ r; rounds run in the order r_t = x^t of
GF(2^5) = GF(2)[x] / (x^5 + x^2 + 1).  At the start of a loop body (round t0),
register k of lane i holds column i ^ (k * x^t0); a body of U rounds is
followed by the renaming k -> k * x^U."""
import itertools

import pytest


def mulx(v):
    return ((v << 1) & 31) ^ (5 if v & 16 else 0)


def gmul(a, b):
    r = 0
    for i in range(5):
        if b & (1 << i):
            r ^= a
        a = mulx(a)
    return r


def gpow(s):
    v = 1
    for _ in range(s):
        v = mulx(v)
    return v


def test_round_order_visits_every_round_once():
    seq = [gpow(t) for t in range(31)]
    assert sorted(seq) == list(range(1, 32))     # x is primitive: order 31
    assert gpow(31) == 1


def test_gf_multiplication_is_a_field_product():
    # commutative, distributive over XOR, and every non-zero element invertible
    for a, b in itertools.product(range(32), repeat=2):
        assert gmul(a, b) == gmul(b, a)
    for a, b, c in [(3, 7, 12), (31, 17, 5), (9, 26, 30)]:
        assert gmul(a, b ^ c) == gmul(a, b) ^ gmul(a, c)
    for a in range(1, 32):
        assert sorted(gmul(a, b) for b in range(32)) == list(range(32))


def test_rounds_are_perfect_matchings_covering_every_pair_once():
    seen = set()
    for r in range(1, 32):
        pairs = {tuple(sorted((i, i ^ r))) for i in range(32)}
        assert len(pairs) == 16                          # disjoint, all 32 indices
        assert not (pairs & seen)
        seen |= pairs
    assert len(seen) == 32 * 31 // 2


@pytest.mark.parametrize("U", [4, 8, 31])
def test_skewed_layout_constants_and_renaming(U):
    """For every lane and round of a body: the diagonal is register 0, the
    pair element is register x^s, the rotated column pairs are the register
    pairs (k, k ^ x^s), and the partner lane keeps this lane's column of
    register k in register k ^ x^s.  The renaming after U rounds gives the
    next body's layout."""
    t0 = 0
    for body in range(40):                       # past several wrap-arounds of t0
        base = gpow(t0 % 31)
        for s in range(U):
            g = gpow(s)
            r = gmul(g, base)
            assert r == gpow((t0 + s) % 31)
            for i in range(32):
                col = [i ^ gmul(k, base) for k in range(32)]
                assert sorted(col) == list(range(32))    # a bijection per lane
                assert col[0] == i                        # diagonal
                assert col[g] == i ^ r                    # pair element
                partner = i ^ r
                pcol = [partner ^ gmul(k, base) for k in range(32)]
                for k in range(32):
                    assert col[k ^ g] == col[k] ^ r        # rotated column pair
                    assert pcol[k ^ g] == col[k]           # partner's copy of my column
        t0 += U
        new_base = gpow(t0 % 31)
        for k in range(32):
            # new register k holds old register k * x^U
            assert gmul(k, new_base) == gmul(gmul(k, gpow(U % 31)), base)
