"""Pins of the oracle's field arithmetic and hash families (Definition 2.1,
Section 2.4, and the Mersenne-prime polynomial hashing named in Section 4)."""
import random

import numpy as np
import pytest

import oracle as O

P = O.P61


def _pow(a, e):
    r, b = 1, a
    while e:
        if e & 1:
            r = O.lib().or_mulmod(r, b)
        b = O.lib().or_mulmod(b, b)
        e >>= 1
    return r


def test_field_map_closed_forms():
    # (uint64)key mod (2^61 - 1); 2^61 = 1 and 2^64 = 8 modulo p
    assert O.field(0) == 0
    assert O.field(P) == 0
    assert O.field(P + 5) == 5
    assert O.field(1 << 61) == 1
    assert O.field(-1) == 7                 # 2^64 - 1
    assert O.field((1 << 63) - 1) == 3      # 2^63 - 1 = 4 - 1
    assert O.field(-(1 << 63)) == 4         # 2^63
    assert O.field(-2) == 6


def test_mulmod_fermat_and_inverse():
    rng = random.Random(1)
    for _ in range(200):
        a = rng.randrange(1, P)
        assert _pow(a, P - 1) == 1                       # Fermat, p prime
        assert O.lib().or_mulmod(a, _pow(a, P - 2)) == 1  # multiplicative inverse
    for a, b in [(P - 1, P - 1), (0, P - 1), (1, P - 1), ((1 << 61) - 2, 2)]:
        assert O.lib().or_mulmod(a, b) == (a * b) % P


def test_poly_monomials_and_linearity():
    rng = random.Random(2)
    for _ in range(100):
        x = rng.randrange(P)
        for t in range(4):
            c = [0, 0, 0, 0]
            c[t] = 1
            assert O.poly(c, x) == _pow(x, t)
        c1 = [rng.randrange(P) for _ in range(4)]
        c2 = [rng.randrange(P) for _ in range(4)]
        s = [(u + v) % P for u, v in zip(c1, c2)]
        assert O.poly(s, x) == (O.poly(c1, x) + O.poly(c2, x)) % P


def test_poly_lagrange_degree3():
    """A degree-3 polynomial is fixed by 4 points: the value at a fifth point equals the
    Lagrange interpolant (inverses by Fermat)."""
    rng = random.Random(3)
    for _ in range(50):
        c = [rng.randrange(P) for _ in range(4)]
        xs = [rng.randrange(P) for _ in range(5)]
        if len(set(xs)) < 5:
            continue
        ys = [O.poly(c, x) for x in xs]
        x5 = xs[4]
        acc = 0
        for i in range(4):
            num, den = 1, 1
            for j in range(4):
                if j != i:
                    num = num * ((x5 - xs[j]) % P) % P
                    den = den * ((xs[i] - xs[j]) % P) % P
            acc = (acc + ys[i] * num * _pow(den, P - 2)) % P
        assert acc == ys[4]


def test_bin_and_sign_ranges():
    rng = random.Random(4)
    for m in [1, 2, 5, 256, 1 << 20, 1000003]:
        for _ in range(50):
            b = np.array([rng.randrange(P), rng.randrange(P)], dtype=np.uint64)
            x = rng.randrange(P)
            v = O.lib().or_bin(b.ctypes.data, x, m)
            assert 0 <= v < m
            assert v == ((int(b[1]) * x + int(b[0])) % P) % m
    s = np.array([rng.randrange(P) for _ in range(4)], dtype=np.uint64)
    assert O.lib().or_sign(s.ctypes.data, 12345) in (-1, 1)
    zero = np.zeros(4, dtype=np.uint64)
    assert O.lib().or_sign(zero.ctypes.data, 999) == 1  # 0 is even


def test_coefficients_in_field_and_deterministic():
    c1 = O.draw_coefficients(42, 3, 2, 3)
    c2 = O.draw_coefficients(42, 3, 2, 3)
    assert c1.shape == (3, 2 * 2 + 4 * 3)
    assert (c1 == c2).all()
    assert (c1 < np.uint64(P)).all()
    c3 = O.draw_coefficients(43, 3, 2, 3)
    assert (c1 != c3).any()


def test_splitmix64_published_vector():
    """First outputs of SplitMix64 seeded with 1234567 as listed in the reference
    implementation's documentation (Vigna, splitmix64.c): 6457827717110365317, 3203168211198807973."""
    st = 1234567
    st, a = O.splitmix64(st)
    st, b = O.splitmix64(st)
    assert a == 6457827717110365317
    assert b == 3203168211198807973


def _sign_of(coeffs_row, x):
    c = np.ascontiguousarray(coeffs_row, dtype=np.uint64)
    return O.lib().or_sign(c.ctypes.data, x)


def _bin_of(coeffs_row, x, m):
    c = np.ascontiguousarray(coeffs_row, dtype=np.uint64)
    return O.lib().or_bin(c.ctypes.data, x, m)


def test_sign_family_pairwise_and_fourwise_moments():
    """E[s(a) s(b)] = 1(a = b) (proof of Theorem 2.3) and, for four distinct keys,
    E[s(a) s(b) s(c) s(e)] = 0 (4-wise independence); checked over N independent draws
    within 4 standard errors (each product is +-1, so the standard error is 1/sqrt(N))."""
    N = 20000
    co = O.draw_coefficients(7, N, 0, 1)  # one sign function per row
    keys = [3, 17, 1 << 40, 999_999_937]
    s = np.array([[_sign_of(co[i], k) for k in keys] for i in range(N)], dtype=np.int64)
    tol = 4.0 / np.sqrt(N)
    for i in range(4):
        for j in range(i + 1, 4):
            assert abs(np.mean(s[:, i] * s[:, j])) < tol
    assert abs(np.mean(s[:, 0] * s[:, 1] * s[:, 2] * s[:, 3])) < tol
    assert abs(np.mean(s[:, 0] * s[:, 1] * s[:, 2])) < tol
    assert abs(np.mean(s[:, 0])) < tol


def test_bin_family_uniform_and_pairwise():
    """A 2-wise independent bin function is uniform on [m] and two distinct keys collide
    with probability 1/m (Definition 2.1)."""
    N, m = 20000, 16
    co = O.draw_coefficients(11, N, 1, 0)
    h1 = np.array([_bin_of(co[i], 5, m) for i in range(N)])
    h2 = np.array([_bin_of(co[i], 123456789, m) for i in range(N)])
    counts = np.bincount(h1, minlength=m)
    chi2 = float(((counts - N / m) ** 2 / (N / m)).sum())
    assert chi2 < 45.0  # chi-square, 15 dof: P(> 45) < 1e-4
    coll = float(np.mean(h1 == h2))
    se = np.sqrt((1 / m) * (1 - 1 / m) / N)
    assert abs(coll - 1 / m) < 4 * se
