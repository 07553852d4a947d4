"""Plain definitions of the space-time FMM pieces (oracle, TEST
INFRASTRUCTURE ONLY).

So far: the coefficients c_m^p(k) of the O(Nt) M2L recurrence (Formula 1,
Eq. cmp) and n_d, the number of auxiliary local coefficients (Remark aux).
"""

from math import comb


def cmp(p, m, k):
    """Eq. (cmp): C(p, m) ((k-1)^{p-m} - 2 k^{p-m} + (k+1)^{p-m}) (-1)^m."""
    e = p - m
    return comb(p, m) * ((k - 1) ** e - 2 * k ** e + (k + 1) ** e) * (-1) ** m


def n_aux(d):
    """Remark aux: n_d = sum_{p=2}^{d} (p - 1)."""
    return sum(p - 1 for p in range(2, d + 1))
