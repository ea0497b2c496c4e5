"""A float32 model of the backprojector's cell walk (the z-profile of one
candidate column, k_backproject.cu), checked on the CPU.

The kernel takes the detector rows of a column in order through the unit
cells kfirst - 1 .. kfirst + VPL - 1 of a lane's voxels. It holds at most C
rows per cell, and it skips the clamp when the first row lo satisfies
lo + (VPL * ntap + 1) / 2 + 2 <= nv + RT_PAD - ntap (2x2-group kernel) or
lo + floor(VPL * rows per voxel) + 2 <= nv + RT_PAD - ntap (one-column
kernel). This model repeats the
walk's float32 arithmetic and row bookkeeping, and checks three things:

* every row it reads lies within both bounds, so the clamp-free loads stay
  inside the zero-padded residual rows;
* its profile equals the direct sum of the interpolation weights
  max(0, 1 - |q_z - k|) r over all rows (the transpose of K1's linear
  interpolation along z), to FP32 rounding;
* it takes every row in the lane's range exactly once.

The row spacings include values within 2e-4 of 1/n, where the choice of C
changes. Host-side check of device index arithmetic; no GPU.
"""
import numpy as np
import pytest

f32 = np.float32
RT_PAD = 8


def fma(a, b, c):
    """fmaf to within a double rounding (the product is exact in float64)."""
    return f32(float(a) * float(b) + float(c))


def ntap_of(inv):
    return int(np.floor(2.0 * float(inv) * 1.0001 + 0.002)) + 1


def cells_rows(inv):
    return int(f32(f32(inv * f32(1.0001)) + f32(0.001))) + 1


def rows_per_cell(step, ntap, inv):
    """The kernel's dispatch: C = 1 when rows are more than a voxel apart,
    else the geometry's bound (ntap + 1) / 2 or one less."""
    cm = (ntap + 1) // 2
    cm1 = cm - 1 if cm > 2 else 2
    if cm < 2 or step > 1:
        return 1
    if cm > 2 and cells_rows(inv) <= cm1:
        return cm1
    return max(cm, 2)


def walk(rows, lo, d0, step, vpl, C):
    """Profile of voxels 0..vpl-1 and the rows read, as the kernel forms them."""
    e = f32(d0 + f32(1))
    prof = np.zeros(vpl, dtype=f32)
    carry = f32(0)
    read = []
    taken = []
    for c in range(vpl + 1):
        v, rv, et = [], [], []
        for t in range(C):
            e_t = e if t == 0 else fma(t, step, e)
            ok = True if (t == 0 and C > 1) else bool(e_t < f32(1))
            read.append(lo + t)
            v.append(ok)
            et.append(e_t)
            rv.append(rows[lo + t] if ok else f32(0))
        s0 = rv[0]
        s1 = f32(et[0] * rv[0])
        for t in range(1, C):
            s0 = f32(s0 + rv[t])
            s1 = fma(et[t], rv[t], s1)
        if c >= 1:
            prof[c - 1] = f32(carry + f32(s0 - s1))
        carry = s1
        if c == vpl:
            break
        en = fma(C, step, e)
        for t in range(C - 1, -1, -1):
            if not v[t]:
                en = e if t == 0 else fma(t, step, e)
        e = f32(en - f32(1))
        n = sum(v)
        taken.extend(range(lo, lo + n))
        lo += n
    return prof, read, taken


@pytest.mark.parametrize("vpl", [2, 4, 8, 16])
def test_cell_walk_bounds_and_values(vpl):
    rng = np.random.default_rng(100 + vpl)
    worst_err, worst_margin = 0.0, -10**9
    for trial in range(3000):
        if trial % 5 == 0:
            n = int(rng.integers(1, 4))
            step = f32(1.0 / n * (1 + rng.uniform(-2e-4, 2e-4)))
        else:
            step = f32(rng.uniform(0.3, 2.5))
        inv = f32(f32(1) / step)
        ntap = ntap_of(inv)
        if ntap > RT_PAD:
            continue
        C = rows_per_cell(step, ntap, inv)
        d0 = f32(-1 + rng.uniform(0, 1) * step)
        if trial % 17 == 0:
            d0 = f32(-1 + step)
        rows = rng.standard_normal(4 * vpl + 64).astype(f32)
        prof, read, taken = walk(rows, 0, d0, step, vpl, C)
        # reads against the clamp-free bounds, relative to the first row: the
        # 2x2-group kernel's (from the geometry's ntap) and the one-column
        # kernel's (from the column's own rows per voxel), both minus ntap - 1
        bound = (vpl * ntap + 1) // 2 + 2 + ntap - 1
        bound1 = int(f32(f32(vpl) * inv)) + 2 + ntap - 1
        worst_margin = max(worst_margin, max(read) - min(bound, bound1))
        assert max(read) <= min(bound, bound1), (step, d0, vpl, C, max(read), bound, bound1)
        assert min(read) >= 0
        # every row of the walk's range taken once, in order
        assert taken == list(range(len(taken)))
        # values against the direct sums of the interpolation weights
        ref = np.zeros(vpl)
        for q in range(vpl):
            for t in range(len(rows)):
                d = float(d0) + t * float(step) - q
                ref[q] += max(0.0, 1.0 - abs(d)) * float(rows[t])
        err = float(np.abs(prof - ref).max() / np.abs(rows).max())
        worst_err = max(worst_err, err)
    assert worst_err < 4e-6, worst_err
    assert worst_margin <= 0
