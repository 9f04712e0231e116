"""CPU pin of the FP32 SpMM's summation, independent of the GPU code: the order and the
operations by which the kernel adds a row's terms (Section 3.3's Y = A X, one output entry at a
time) are restated in numpy float32 scalars and the kernel's stated worst case per entry,
9 * 2^-24 * sum |x|, is checked against exact sums on inputs chosen to make rounding errors add
up (one sign, constant values, wide exponent ranges, near-total cancellation).

The summation restated:
* a warp task (rows of degree above the slice limit, and every chunk of a split hub row):
  term k of the task goes to slot k mod P (P = 32 / chunks per row: 32 for b <= 4, 32 or 16
  for b = 8 and 16 or 8 for b = 16, by the load width); every slot adds its terms in order with Kahan's compensation (s, c) and ends with
  s - c; the P slot values are added by a balanced tree (slot s with slot s + P/2, then + P/4,
  ...), one FP32 add per level;
* a slice row (the low-degree tail): one lane adds the row's terms in order, compensated;
* a split hub row: its chunks' task results are added in FP64 with Neumaier's compensation in
  task order and rounded once to FP32.
Bound: 3 u per slot (2 u + O(m u^2) for the compensated sum, Higham Thm. 4.8, plus the rounding
of s - c), u per tree level (at most 5), u for the hub's final rounding: 9 u with u = 2^-24.
"""
import math

import numpy as np
import pytest

F = np.float32
U = 2.0 ** -24
BOUND = 9 * U


def slot_sum(terms):
    """Kahan's compensated sum of float32 terms in order, then s - c (float32 throughout)."""
    s = F(0.0)
    c = F(0.0)
    for x in terms:
        y = F(x - c)
        t = F(s + y)
        c = F((t - s) - y)
        s = t
    return F(s - c)


def plain_slot_sum(terms):
    """The same slot without compensation (what an uncompensated kernel computes)."""
    s = F(0.0)
    for x in terms:
        s = F(s + x)
    return s


def task_sum(terms, P, slot=slot_sum):
    """One warp task: slot k mod P, compensated slot sums, then a balanced tree over slots."""
    part = [slot(terms[s::P]) for s in range(P)]
    h = P // 2
    while h >= 1:
        part = [F(part[s] + part[s + h]) for s in range(h)]
        h //= 2
    return part[0]


def hub_sum(terms, task_len, P):
    """A split hub row: task results in FP64 with Neumaier's compensation, rounded once."""
    s = e = 0.0
    for t0 in range(0, len(terms), task_len):
        x = float(task_sum(terms[t0:t0 + task_len], P))
        u = s + x
        e += (s - u) + x if abs(s) >= abs(x) else (x - u) + s
        s = u
    return F(s + e)


def rel_err(got, terms):
    """|got - exact sum| / sum |x| (0 for an all-zero row, which must come out exactly 0)."""
    exact = math.fsum(float(t) for t in terms)
    scale = math.fsum(abs(float(t)) for t in terms)
    if scale == 0.0:
        return 0.0 if float(got) == 0.0 else math.inf
    return abs(float(got) - exact) / scale


def adversarial_rows(rng, deg):
    """Rows of `deg` float32 terms that make rounding errors add up."""
    rows = {
        "const": np.full(deg, F(1.9397392272949219), dtype=F),
        "u12": (1.0 + rng.random(deg)).astype(F),
        "u01": rng.random(deg).astype(F),
        "wide": (rng.choice([-1.0, 1.0], deg) * 10.0 ** rng.uniform(-8, 8, deg)).astype(F),
        "geom": (1.0 + 2.0 ** -rng.integers(1, 24, deg)).astype(F),
    }
    cancel = rng.standard_normal(deg).astype(F)                 # sum ~ 0 relative to sum |x|
    cancel[-1] = F(-math.fsum(float(t) for t in cancel[:-1]))
    rows["cancel"] = cancel
    big = np.full(deg, F(1.0 + 2.0 ** -23), dtype=F)
    big[0] = F(2.0 ** 20)                                       # one large term first
    rows["big_first"] = big
    return rows


@pytest.mark.parametrize("P", [32, 16, 8])
@pytest.mark.parametrize("deg", [1, 31, 33, 127, 128, 500, 3000])
def test_warp_task_within_bound(P, deg):
    rng = np.random.default_rng(1000 * P + deg)
    for name, terms in adversarial_rows(rng, deg).items():
        err = rel_err(task_sum(terms, P), terms)
        assert err <= BOUND, (name, P, deg, err / U)


@pytest.mark.parametrize("deg", [1, 2, 17, 69, 127, 128])
def test_slice_row_within_bound(deg):
    rng = np.random.default_rng(deg)
    for name, terms in adversarial_rows(rng, deg).items():
        err = rel_err(slot_sum(terms), terms)
        assert err <= BOUND, (name, deg, err / U)


@pytest.mark.parametrize("P", [32, 8])
def test_split_hub_row_within_bound(P):
    rng = np.random.default_rng(7 + P)
    deg, task_len = 20000, 4096                                 # five chunks, the last ragged
    for name, terms in adversarial_rows(rng, deg).items():
        err = rel_err(hub_sum(terms, task_len, P), terms)
        assert err <= BOUND, (name, P, err / U)


def test_uncompensated_sums_exceed_the_bound():
    """The pin is sensitive: the same orders without compensation exceed 9 u on one-signed
    rows -- a slice row of degree 127 and a long warp task -- so a kernel that lost the
    compensation would be caught by the GPU tests' inputs."""
    const127 = np.full(127, F(1.9397392272949219), dtype=F)
    assert rel_err(plain_slot_sum(const127), const127) > 1e-6 > BOUND
    long_row = np.full(32 * 256, F(1.9397392272949219), dtype=F)   # 256 terms per slot
    assert rel_err(task_sum(long_row, 32, plain_slot_sum), long_row) > BOUND
    assert rel_err(task_sum(long_row, 32), long_row) <= BOUND
