"""Pins of the oracle's M2L recurrence constants against the paper's table
(Remark on c_m^p(k), Section 4.3) and Remark aux (n_d)."""

import os

import numpy as np

from oracle import fmm

GOLD = os.path.join(os.path.dirname(__file__), "golden")


def test_cmp_matches_printed_table():
    for line in open(os.path.join(GOLD, "table_cmp.txt")):
        if line.startswith("#") or not line.strip():
            continue
        key, poly = line.split(":")
        p, m = map(int, key.split())
        coef = [int(c) for c in poly.split()]
        for k in range(-3, 7):
            assert fmm.cmp(p, m, k) == sum(c * k ** e for e, c in enumerate(coef))


def test_cmp_vanishes_for_m_ge_p_minus_1():
    for p in range(1, 7):
        for k in range(-2, 5):
            assert fmm.cmp(p, p, k) == 0
            if p >= 1:
                assert fmm.cmp(p, p - 1, k) == 0


def test_cmp_is_second_difference_expansion():
    # (k-1-l)^p - 2 (k-l)^p + (k+1-l)^p = sum_m c_m^p(k) l^m  (Eq. tmp1)
    for p in range(2, 6):
        for k in range(0, 5):
            for l in range(-2, 6):
                lhs = (k - 1 - l) ** p - 2 * (k - l) ** p + (k + 1 - l) ** p
                assert lhs == sum(fmm.cmp(p, m, k) * l ** m for m in range(0, p - 1))


def test_n_aux():
    assert [fmm.n_aux(d) for d in range(1, 6)] == [0, 1, 3, 6, 10]
