"""The kernels step Dormand-Prince 5(4) in second-order (Nystrom) form with
coefficients derived from the published tableau (Dormand & Prince 1980):
abar_sk = sum_j a_sj a_jk, bbar_k = sum_j b_j a_jk, ehat_k = sum_j E_j a_jk.
This test re-derives them in exact rational arithmetic from the tableau
written out here and compares them with the constants in the CUDA source,
so a typo in any derived coefficient is caught without a GPU."""
import os
import re
from fractions import Fraction as Fr

SRC = os.path.join(os.path.dirname(__file__), "..", "paper_2507_16165_gb300", "csrc", "tracer.cuh")

# Dormand & Prince (1980), RK5(4)7M: a_sj, fifth-order weights b_j and the
# fourth-order weights bhat_j
A = {(2, 1): Fr(1, 5),
     (3, 1): Fr(3, 40), (3, 2): Fr(9, 40),
     (4, 1): Fr(44, 45), (4, 2): Fr(-56, 15), (4, 3): Fr(32, 9),
     (5, 1): Fr(19372, 6561), (5, 2): Fr(-25360, 2187), (5, 3): Fr(64448, 6561),
     (5, 4): Fr(-212, 729),
     (6, 1): Fr(9017, 3168), (6, 2): Fr(-355, 33), (6, 3): Fr(46732, 5247), (6, 4): Fr(49, 176),
     (6, 5): Fr(-5103, 18656)}
B = {1: Fr(35, 384), 2: Fr(0), 3: Fr(500, 1113), 4: Fr(125, 192), 5: Fr(-2187, 6784),
     6: Fr(11, 84), 7: Fr(0)}
BHAT = {1: Fr(5179, 57600), 2: Fr(0), 3: Fr(7571, 16695), 4: Fr(393, 640),
        5: Fr(-92097, 339200), 6: Fr(187, 2100), 7: Fr(1, 40)}
for j in range(1, 7):
    A[(7, j)] = B[j]           # the seventh stage is the fifth-order solution


def a(s, j):
    return A.get((s, j), Fr(0))


def kernel_constants() -> dict:
    text = open(SRC).read()
    out = {}
    for name, num, den in re.findall(r"#define DP_(\w+) \((-?\d+)\.0 / (\d+)\.0\)", text):
        out[name] = Fr(int(num), int(den))
    return out


def test_nystrom_coefficients_follow_from_the_tableau():
    k = kernel_constants()
    E = {j: B[j] - BHAT[j] for j in range(1, 8)}
    assert sum(E.values()) == 0            # why e_u has no h v term
    for s in (2, 3, 4, 5):
        assert k[f"C{s}"] == sum(a(s, j) for j in range(1, s))
    assert sum(a(6, j) for j in range(1, 6)) == 1   # c_6 = 1: the kernel adds h v
    for s, ks in ((3, (1,)), (4, (1, 2)), (5, (1, 2, 3)), (6, (1, 2, 3, 4))):
        for kk in range(1, s):
            abar = sum(a(s, j) * a(j, kk) for j in range(1, s))
            if kk in ks:
                assert k[f"AB{s}{kk}"] == abar, (s, kk)
            else:
                assert abar == 0, (s, kk)     # left out of the kernel
    for kk in range(1, 7):
        bbar = sum(B[j] * a(j, kk) for j in range(1, 7))
        if f"BB{kk}" in k:
            assert k[f"BB{kk}"] == bbar, kk
        else:
            assert bbar == 0, kk
        ehat = sum(E[j] * a(j, kk) for j in range(2, 8))
        if f"EH{kk}" in k:
            assert k[f"EH{kk}"] == ehat, kk
        else:
            assert ehat == 0, kk
        if B[kk] != 0:
            assert k[f"B{kk}"] == B[kk]
    for j in range(1, 8):
        if E[j] != 0:
            assert k[f"E{j}"] == E[j], j


def test_nystrom_step_equals_first_order_step_exactly():
    """One step of both forms in exact arithmetic on a polynomial right-hand
    side gives identical results (they are the same method)."""
    k = kernel_constants()
    M3 = Fr(3)
    F = lambda u: u * (M3 * u - 1)
    u, v, h = Fr(1, 50), Fr(-1, 30), Fr(3, 10)
    # first-order form
    V = {1: v}
    Fs = {1: F(u)}
    for s in range(2, 8):
        U = u + h * sum(a(s, j) * V[j] for j in range(1, s))
        V[s] = v + h * sum(a(s, j) * Fs[j] for j in range(1, s))
        Fs[s] = F(U)
    un1 = u + h * sum(B[j] * V[j] for j in range(1, 7))
    vn1 = V[7]
    E = {j: B[j] - BHAT[j] for j in range(1, 8)}
    eu1 = h * sum(E[j] * V[j] for j in range(1, 8))
    ev1 = h * sum(E[j] * Fs[j] for j in range(1, 8))
    # Nystrom form with the kernel's constants
    hv, h2 = h * v, h * h
    f1 = F(u)
    F2 = F(u + k["C2"] * hv)
    F3 = F(u + k["C3"] * hv + h2 * k["AB31"] * f1)
    F4 = F(u + k["C4"] * hv + h2 * (k["AB41"] * f1 + k["AB42"] * F2))
    F5 = F(u + k["C5"] * hv + h2 * (k["AB51"] * f1 + k["AB52"] * F2 + k["AB53"] * F3))
    F6 = F(u + hv + h2 * (k["AB61"] * f1 + k["AB62"] * F2 + k["AB63"] * F3 + k["AB64"] * F4))
    un = u + hv + h2 * (k["BB1"] * f1 + k["BB3"] * F3 + k["BB4"] * F4 + k["BB5"] * F5)
    vn = v + h * (k["B1"] * f1 + k["B3"] * F3 + k["B4"] * F4 + k["B5"] * F5 + k["B6"] * F6)
    fn = F(un)
    eu = h2 * (k["EH1"] * f1 + k["EH3"] * F3 + k["EH4"] * F4 + k["EH5"] * F5 + k["EH6"] * F6)
    ev = h * (k["E1"] * f1 + k["E3"] * F3 + k["E4"] * F4 + k["E5"] * F5 + k["E6"] * F6
              + k["E7"] * fn)
    assert (un, vn, eu, ev) == (un1, vn1, eu1, ev1)
