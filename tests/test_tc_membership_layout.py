"""The term layout of the tensor-core sub-horizon membership test (mixed
path), restated on the host with numpy: each scaled bond-vector component and
|zeta~|^2 split into two fp16 terms (a Veltkamp split in FP32, the high part
exact in fp16, the low part rounded to fp16), products of the bond row and the
member column summed exactly (float64 here; the tensor cores sum the same
exact fp16 products in FP32), plus the bond's start term e_t = sT^2 (|zeta~_t|^2
- hf^2) either as an FP32 accumulator start (the warp kernel) or as two more
split terms (the tensor-memory kernel).

Checked against the exact squared distances |zeta~_k - zeta~_t|^2 - hf^2 of
FP32 bond vectors on perturbed lattice families: the error stays near 1e-6
of hf^2 (below 1.5e-6) and every pair farther than that from the sub-horizon
radius is decided as the exact test decides it, which is the precision the design
claims for this test (an FP32-class rounding).  No GPU is used.
"""
import itertools

import numpy as np
import pytest

F32, F16 = np.float32, np.float16


def split(x):
    """Veltkamp split with 2^13 + 1 in FP32, then both parts in fp16."""
    x = np.asarray(x, F32)
    c = (x * F32(8193)).astype(F32)
    hi = (c - (c - x).astype(F32)).astype(F32)
    lo = (x - hi).astype(F32)
    return hi.astype(F16).astype(np.float64), lo.astype(F16).astype(np.float64)


def scale_of(m):
    """2^-(e+1) for 2^e <= m < 2^(e+1)."""
    e = (np.float32(m).view(np.uint32) >> 23) & 0xFF
    return F32(1.0) if (e == 0 or e >= 253) else np.uint32((253 - e) << 23).view(F32)


def family(perturb, seed, horizon=3.015):
    offs = np.array([o for o in itertools.product(range(-3, 4), repeat=3)
                     if 0 < o[0] ** 2 + o[1] ** 2 + o[2] ** 2 <= horizon ** 2], np.float64)
    rng = np.random.default_rng(seed)
    return (offs + rng.uniform(-perturb, perturb, offs.shape)).astype(F32)


def tc_distances(z, hf2, start_in_accumulator):
    z = np.asarray(z, F32)
    w = (z[:, 0] * z[:, 0] + z[:, 1] * z[:, 1] + z[:, 2] * z[:, 2]).astype(F32)
    sT = scale_of(np.abs(z).max())
    sT2 = F32(sT * sT)
    hf2s = F32(F32(hf2) * sT2)
    cs = (z * sT).astype(F32)
    ws = (w * sT2).astype(F32)
    e = (ws.astype(np.float64) - np.float64(hf2s)).astype(F32)   # one FP32 rounding, as the FMA
    d = np.zeros((len(z), len(z)))
    for c in range(3):
        h, l = split(cs[:, c])
        # bond row (-2c^h, -2c^h, -2c^l, -2c^l) against member column (c^h, c^l, c^h, c^l)
        d += np.outer(-2 * h, h) + np.outer(-2 * h, l) + np.outer(-2 * l, h) + np.outer(-2 * l, l)
    wh, wl = split(ws)
    d += (wh + wl)[None, :]
    if start_in_accumulator:
        d += e.astype(np.float64)[:, None]
    else:
        eh, el = split(e)
        d += (eh + el)[:, None]
    return d / np.float64(sT2)


@pytest.mark.parametrize("perturb,seed", [(0.05, 1), (0.3, 2), (0.6, 3)])
@pytest.mark.parametrize("start_in_accumulator", [True, False])
def test_tensor_core_test_is_fp32_class(perturb, seed, start_in_accumulator):
    hf = 3.015 * 0.83                       # a sub-horizon radius in lattice units
    hf2 = np.float64(F32(hf * hf))
    z = family(perturb, seed)
    zd = z.astype(np.float64)
    exact = ((zd[None, :, :] - zd[:, None, :]) ** 2).sum(-1) - hf2
    d = tc_distances(z, hf2, start_in_accumulator)
    err = np.abs(d - exact)
    assert err.max() <= 1.5e-6 * hf2, err.max() / hf2
    clear = np.abs(exact) > 1.5e-6 * hf2
    assert np.array_equal((d < 0)[clear], (exact < 0)[clear])
    # the layout is not trivially exact: the low parts carry real information
    assert err.max() > 0.0


def test_a_bond_is_in_its_own_sub_horizon_and_far_members_are_not():
    z = family(0.2, 7)
    hf2 = np.float64(F32(2.5 ** 2))
    d = tc_distances(z, hf2, True)
    assert np.all(np.diag(d) < 0)
    zd = z.astype(np.float64)
    exact = ((zd[None, :, :] - zd[:, None, :]) ** 2).sum(-1) - hf2
    assert np.all(d[exact > 1.0] > 0)
