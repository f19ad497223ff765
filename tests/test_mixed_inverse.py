"""The mixed path's shape-tensor inverse, restated on the host in exact
rational arithmetic with binary32 rounding (round to nearest even) at each
step the kernel rounds: the tensor scaled by a power of two into [1, 2), the
determinant from FP64 cofactors (taken exact here: FP64 carries it to about
1e-16 times the condition number, far below the binary32 rounding that
follows), rounded once to binary32; its correctly rounded reciprocal; each
entry a 2 x 2 minor by Kahan's FMA algorithm (w = RN(c d), e = RN(w - c d)
which is exact, f = RN(a b - w), RN(f + e)) times that reciprocal.

Pinned against the exact inverse of the same binary32 tensor: every entry
within 4 ulp-units (4 * 2^-24) of its exact value, relative to that entry,
for well- and ill-conditioned tensors (condition numbers to 1e6) and for
shape tensors of perturbed lattice sub-horizons.  Kahan's minor alone is
held to its published bound (relative error at most 2 * 2^-24) on
cancelling inputs.  No GPU is used."""
from fractions import Fraction as Q
import itertools

import numpy as np
import pytest

F32 = np.float32
U = Q(1, 2 ** 24)


def rn32(x: Q) -> Q:
    """x rounded to the nearest binary32 number (ties to even), as a Fraction."""
    if x == 0:
        return Q(0)
    f = np.float32(float(x))
    best = None
    for c in (f, np.nextafter(f, F32(np.inf)), np.nextafter(f, F32(-np.inf))):
        d = abs(Q(float(c)) - x)
        odd = int(np.array(c, F32).view(np.uint32)) & 1
        key = (d, odd)
        if best is None or key < best[0]:
            best = (key, c)
    return Q(float(best[1]))


def minor2(a: Q, b: Q, c: Q, d: Q) -> Q:
    """a b - c d of binary32 numbers by Kahan's algorithm."""
    w = rn32(c * d)
    e = rn32(w - c * d)            # the FMA: exact, the rounding error of c d
    f = rn32(a * b - w)            # the FMA
    return rn32(f + e)


def mixed_inverse(K):
    """K = (xx, yy, zz, yz, xz, xy) binary32; the inverse in the same order."""
    k = [Q(float(F32(v))) for v in K]
    m = max(abs(v) for v in k)
    e = int(np.floor(np.log2(float(m))))
    sc = Q(2) ** (-e)               # the largest |entry| scaled into [1, 2)
    s00, s11, s22, s12, s02, s01 = (v * sc for v in k)
    c00 = s11 * s22 - s12 * s12
    c01 = s02 * s12 - s01 * s22
    c02 = s01 * s12 - s02 * s11
    det = rn32(s00 * c00 + s01 * c01 + s02 * c02)
    r = rn32(1 / det) * sc
    minors = (minor2(s11, s22, s12, s12), minor2(s00, s22, s02, s02), minor2(s00, s11, s01, s01),
              minor2(s01, s02, s00, s12), minor2(s01, s12, s02, s11), minor2(s02, s12, s01, s22))
    return [rn32(mm * r) for mm in minors]


def exact_inverse(K):
    k00, k11, k22, k12, k02, k01 = (Q(float(F32(v))) for v in K)
    M = [[k00, k01, k02], [k01, k11, k12], [k02, k12, k22]]
    det = (M[0][0] * (M[1][1] * M[2][2] - M[1][2] * M[2][1])
           - M[0][1] * (M[1][0] * M[2][2] - M[1][2] * M[2][0])
           + M[0][2] * (M[1][0] * M[2][1] - M[1][1] * M[2][0]))
    adj = {
        (0, 0): M[1][1] * M[2][2] - M[1][2] * M[1][2],
        (1, 1): M[0][0] * M[2][2] - M[0][2] * M[0][2],
        (2, 2): M[0][0] * M[1][1] - M[0][1] * M[0][1],
        (1, 2): M[0][1] * M[0][2] - M[0][0] * M[1][2],
        (0, 2): M[0][1] * M[1][2] - M[0][2] * M[1][1],
        (0, 1): M[0][2] * M[1][2] - M[0][1] * M[2][2],
    }
    order = [(0, 0), (1, 1), (2, 2), (1, 2), (0, 2), (0, 1)]
    return [adj[o] / det for o in order], det


def spd(rng, cond, scale):
    A = rng.normal(size=(3, 3))
    Qm, _ = np.linalg.qr(A)
    lam = np.array([1.0, cond ** rng.uniform(0.2, 0.8), cond]) * scale
    S = Qm @ np.diag(lam) @ Qm.T
    return [S[0, 0], S[1, 1], S[2, 2], S[1, 2], S[0, 2], S[0, 1]]


def lattice_shape_tensor(rng, perturb, radius=2.5, flat=None):
    offs = np.array([o for o in itertools.product(range(-3, 4), repeat=3)
                     if 0 < sum(x * x for x in o) <= radius ** 2], float)
    if flat is not None:                                   # a thin slab of members
        offs = offs[np.abs(offs[:, 2]) <= flat]
    z = (offs + rng.uniform(-perturb, perturb, offs.shape)).astype(F32)
    K = np.zeros(6)
    for a, b, q in ((0, 0, 0), (1, 1, 1), (2, 2, 2), (1, 2, 3), (0, 2, 4), (0, 1, 5)):
        K[q] = float(np.sum(z[:, a].astype(np.float64) * z[:, b]))
    return K


def check(K, tol_units=4):
    got = mixed_inverse(K)
    want, det = exact_inverse(K)
    assert det > 0
    for g, w in zip(got, want):
        assert abs(g - w) <= tol_units * U * abs(w), (float(g), float(w))


def test_kahan_minor_meets_its_bound_on_cancelling_inputs():
    rng = np.random.default_rng(1)
    worst = Q(0)
    for _ in range(3000):
        a, b, c = (Q(float(F32(x))) for x in rng.uniform(0.5, 2.0, 3))
        # d chosen so that c d nearly equals a b: heavy cancellation
        d = Q(float(F32(float(a * b / c) * (1 + rng.normal() * 1e-6))))
        exact = a * b - c * d
        got = minor2(a, b, c, d)
        if exact != 0:
            worst = max(worst, abs(got - exact) / abs(exact))
        else:
            assert got == 0
    assert worst <= 2 * U, float(worst / U)
    assert worst > 0                     # the rounding is real, not vacuous


@pytest.mark.parametrize("cond", [1.0, 1e2, 1e4, 1e6])
def test_random_tensors_invert_to_a_few_ulp_of_each_entry(cond):
    rng = np.random.default_rng(int(cond) % 1000 + 3)
    for q in range(40):
        scale = 2.0 ** rng.integers(-20, 20)
        check(spd(rng, cond, scale))


@pytest.mark.parametrize("perturb,flat", [(0.0, None), (0.05, None), (0.3, None), (0.02, 0.0)])
def test_lattice_sub_horizon_tensors_invert_to_a_few_ulp(perturb, flat):
    # the planar family (flat = 0: members in one lattice plane, slightly
    # perturbed out of it) is the ill-conditioned case of the surfaces
    rng = np.random.default_rng(11)
    for _ in range(10):
        K = lattice_shape_tensor(rng, perturb, flat=flat)
        if flat is not None:
            K = [F32(v) for v in K]
            if exact_inverse(K)[1] <= 0:
                continue
        check(K)


def test_a_minor_without_the_error_term_fails_the_bound():
    # the plausible mistake: RN(RN(a b) - RN(c d)), the error term dropped;
    # on cancelling inputs it is far outside 2u, so the pin above can see it
    rng = np.random.default_rng(1)
    worst = Q(0)
    for _ in range(300):
        a, b, c = (Q(float(F32(x))) for x in rng.uniform(0.5, 2.0, 3))
        d = Q(float(F32(float(a * b / c) * (1 + rng.normal() * 1e-6))))
        exact = a * b - c * d
        naive = rn32(rn32(a * b) - rn32(c * d))
        if exact != 0:
            worst = max(worst, abs(naive - exact) / abs(exact))
    assert worst > 100 * U
