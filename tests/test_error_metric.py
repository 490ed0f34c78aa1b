"""Pins for the oracle's error metric, rel_l2 and rel_l2_rows.

Every GPU parity gate is a bound on these two numbers, so they are checked
against values worked out by hand (not by calling numpy's norm the same way
the functions do), and each plausible slip -- a norm over the wrong axis, a
ratio left squared, a missing square root on one side, a ratio taken against
the result instead of the reference, a max-abs norm instead of L2, the
reference's norm taken row by row in rel_l2 -- is planted in a copy and shown
to fail at least one pin.

The definition being pinned (relative L2 error, the error measure the
configurations state): for a result g and a reference r,
    rel_l2(g, r)      = sqrt(sum |g - r|^2) / sqrt(sum |r|^2) over all elements,
    rel_l2_rows(g, r) = the same ratio for every row (last axis) separately,
and the bare numerator when the reference is all zeros.
"""
from __future__ import annotations

import numpy as np
import pytest

import oracle


# --- hand-worked cases ----------------------------------------------------------
# rel_l2: (got, ref, value) with the value derived by hand beside each.
REL_L2_CASES = [
    # |(3,4) - (0,0)| / |(3,4)| = 5 / 5
    (np.array([0, 0]), np.array([3, 4]), 1.0),
    # one complex value 3+4i (|.| = 5) off by 0.5 in the real part: 0.5 / 5
    (np.array([3.5 + 4j]), np.array([3 + 4j]), 0.1),
    # ref = (1, i, -1, -i): |ref| = 2; got off by 0.1 in one entry: 0.1 / 2
    (np.array([1.1, 1j, -1, -1j]), np.array([1, 1j, -1, -1j]), 0.05),
    # 2x2 array [[3,0],[0,4]] (norm 5) against [[3,0],[0,0]]: error 4, so 4/5;
    # every element counts, whatever the shape
    (np.array([[3, 0], [0, 0]]), np.array([[3, 0], [0, 4]]), 0.8),
    # errors in both parts: ref (6+8i) has norm 10; got (6+8i) + (1+2i)
    # differs by sqrt(1 + 4) = sqrt(5): sqrt(5) / 10
    (np.array([7 + 10j]), np.array([6 + 8j]), np.sqrt(5.0) / 10.0),
    # exact match
    (np.array([1 + 1j, 2]), np.array([1 + 1j, 2]), 0.0),
    # zero reference: the bare numerator |(3,4)| = 5
    (np.array([3, 4]), np.array([0, 0]), 5.0),
]

# rel_l2_rows: (got, ref, per-row values), each row worked by hand.
REL_L2_ROWS_CASES = [
    # row 0: ref (3+4i, 0) norm 5, error 0.5 in the second entry -> 0.1
    # row 1: ref (1, 1) norm sqrt(2), error 1 in the second entry -> 1/sqrt(2)
    (np.array([[3 + 4j, 0.5], [1, 0]]), np.array([[3 + 4j, 0], [1, 1]]), [0.1, 1.0 / np.sqrt(2.0)]),
    # three rows of one element each: |1.5 - 1|/1, |2 - 2|/2, |0 - 4i|/4
    (np.array([[1.5], [2], [0]]), np.array([[1], [2], [4j]]), [0.5, 0.0, 1.0]),
    # a zero reference row gives its bare numerator |(0.3, 0.4)| = 0.5
    (np.array([[0.3, 0.4], [2, 0]]), np.array([[0, 0], [2, 0]]), [0.5, 0.0]),
]


def _rows3d():
    """A (2, 1, 3) array: rows are along the last axis, the leading axes stay."""
    ref = np.array([[[2, 0, 0]], [[0, 0, 5j]]])
    got = np.array([[[2, 1, 0]], [[0, 0, 5j + 2.5]]])
    # row (0,0): error 1 over norm 2 -> 0.5;  row (1,0): error 2.5 over 5 -> 0.5
    return got, ref, np.array([[0.5], [0.5]])


def check_rel_l2(fn):
    for got, ref, want in REL_L2_CASES:
        v = fn(got, ref)
        assert np.isscalar(v) or np.ndim(v) == 0, "rel_l2 returns one number"
        assert abs(float(v) - want) <= 1e-15 * max(1.0, want), f"rel_l2({got}, {ref}) = {v}, by hand {want}"


def check_rel_l2_rows(fn):
    for got, ref, want in REL_L2_ROWS_CASES:
        v = np.asarray(fn(got, ref))
        assert v.shape == (len(want),), f"one value per row, got shape {v.shape}"
        assert np.allclose(v, want, rtol=1e-15, atol=1e-16), f"rel_l2_rows = {v}, by hand {want}"
    got, ref, want = _rows3d()
    v = np.asarray(fn(got, ref))
    assert v.shape == want.shape and np.allclose(v, want, rtol=1e-15, atol=0), f"3-D rows: {v}"


def check_scale_invariance(fn):
    """Scaling result and reference together leaves a relative error alone;
    scaling only the error scales it linearly (not quadratically)."""
    g = np.random.Generator(np.random.PCG64(4))
    ref = g.standard_normal(64) + 1j * g.standard_normal(64)
    err = 1e-3 * (g.standard_normal(64) + 1j * g.standard_normal(64))
    base = float(np.max(fn(ref + err, ref)))
    assert abs(float(np.max(fn(1e6 * (ref + err), 1e6 * ref))) - base) <= 1e-12 * base
    assert abs(float(np.max(fn(ref + 3 * err, ref))) - 3 * base) <= 1e-12 * base


def test_rel_l2_hand_worked():
    check_rel_l2(oracle.rel_l2)


def test_rel_l2_rows_hand_worked():
    check_rel_l2_rows(oracle.rel_l2_rows)


def test_rel_l2_rows_agrees_with_rel_l2_on_each_row():
    """Two independent statements of one definition: the per-row function on
    a batch equals the whole-array function applied to each row alone."""
    g = np.random.Generator(np.random.PCG64(9))
    ref = g.standard_normal((5, 16)) + 1j * g.standard_normal((5, 16))
    got = ref + (10.0 ** -np.arange(5))[:, None] * g.standard_normal((5, 16))
    rows = oracle.rel_l2_rows(got, ref)
    for b in range(5):
        assert abs(rows[b] - oracle.rel_l2(got[b], ref[b])) <= 1e-15 * rows[b]


def test_scale_behaviour():
    check_scale_invariance(oracle.rel_l2)
    check_scale_invariance(oracle.rel_l2_rows)


# --- planted mistakes: each must fail a pin ------------------------------------------
def _wrong_axis_rows(got, ref):
    g, r = np.asarray(got, np.complex128), np.asarray(ref, np.complex128)
    den = np.sqrt(np.sum(np.abs(r) ** 2, axis=0))
    num = np.sqrt(np.sum(np.abs(g - r) ** 2, axis=0))
    return num / np.where(den > 0, den, 1.0)


def _squared_ratio_rows(got, ref):
    g, r = np.asarray(got, np.complex128), np.asarray(ref, np.complex128)
    den = np.sum(np.abs(r) ** 2, axis=-1)
    num = np.sum(np.abs(g - r) ** 2, axis=-1)
    return num / np.where(den > 0, den, 1.0)


def _no_sqrt_num_rows(got, ref):
    g, r = np.asarray(got, np.complex128), np.asarray(ref, np.complex128)
    den = np.sqrt(np.sum(np.abs(r) ** 2, axis=-1))
    num = np.sum(np.abs(g - r) ** 2, axis=-1)
    return num / np.where(den > 0, den, 1.0)


def _against_got_rows(got, ref):
    g, r = np.asarray(got, np.complex128), np.asarray(ref, np.complex128)
    den = np.sqrt(np.sum(np.abs(g) ** 2, axis=-1))
    num = np.sqrt(np.sum(np.abs(g - r) ** 2, axis=-1))
    return num / np.where(den > 0, den, 1.0)


def _maxabs_rows(got, ref):
    g, r = np.asarray(got, np.complex128), np.asarray(ref, np.complex128)
    den = np.max(np.abs(r), axis=-1)
    num = np.max(np.abs(g - r), axis=-1)
    return num / np.where(den > 0, den, 1.0)


def _real_part_only_rows(got, ref):
    g, r = np.asarray(got, np.complex128), np.asarray(ref, np.complex128)
    den = np.sqrt(np.sum(r.real ** 2, axis=-1))
    num = np.sqrt(np.sum((g - r).real ** 2, axis=-1))
    return num / np.where(den > 0, den, 1.0)


def _squared_ratio(got, ref):
    d = np.asarray(got, np.complex128) - np.asarray(ref, np.complex128)
    den = np.sum(np.abs(np.asarray(ref, np.complex128)) ** 2)
    return float(np.sum(np.abs(d) ** 2) / den) if den > 0 else float(np.sum(np.abs(d) ** 2))


def _against_got(got, ref):
    d = np.asarray(got, np.complex128) - np.asarray(ref, np.complex128)
    den = np.linalg.norm(np.asarray(got, np.complex128).reshape(-1))
    return float(np.linalg.norm(d.reshape(-1)) / den) if den > 0 else float(np.linalg.norm(d.reshape(-1)))


def _max_of_rows(got, ref):
    g, r = np.atleast_2d(np.asarray(got, np.complex128)), np.atleast_2d(np.asarray(ref, np.complex128))
    return float(np.max(oracle.rel_l2_rows(g, r)))


def _mean_not_sum(got, ref):
    d = np.abs(np.asarray(got, np.complex128) - np.asarray(ref, np.complex128)).reshape(-1)
    r = np.abs(np.asarray(ref, np.complex128)).reshape(-1)
    den = np.sqrt(np.mean(r ** 2))
    return float(np.sqrt(np.sum(d ** 2)) / den) if den > 0 else float(np.sqrt(np.sum(d ** 2)))


ROW_MUTANTS = {"wrong axis": _wrong_axis_rows, "squared ratio": _squared_ratio_rows,
               "no sqrt in numerator": _no_sqrt_num_rows, "relative to result": _against_got_rows,
               "max-abs norm": _maxabs_rows, "real part only": _real_part_only_rows}
WHOLE_MUTANTS = {"squared ratio": _squared_ratio, "relative to result": _against_got,
                 "max over rows": _max_of_rows, "mean in denominator": _mean_not_sum}


@pytest.mark.parametrize("name", sorted(ROW_MUTANTS))
def test_rows_pins_catch_mutation(name):
    fn = ROW_MUTANTS[name]
    with pytest.raises(AssertionError):
        check_rel_l2_rows(fn)
        check_scale_invariance(fn)


@pytest.mark.parametrize("name", sorted(WHOLE_MUTANTS))
def test_whole_pins_catch_mutation(name):
    fn = WHOLE_MUTANTS[name]
    with pytest.raises(AssertionError):
        check_rel_l2(fn)
        check_scale_invariance(fn)
