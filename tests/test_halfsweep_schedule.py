"""CPU check of the schedule behind the 3-D half-sweep smoother (no GPU).

The 8-colour Gauss-Seidel order (colour (i&1) + 2(j&1) + 4(k&1), Sec. 2.2's
smoother in 3-D) visits every colour of the even k-planes before those of the
odd ones, and planes couple only through z-couplings, which join planes of
opposite parity.  So a sweep splits into two halves, each an independent
4-colour sweep per plane against fixed neighbouring planes, and within a
plane the last colour depends on the first through at most three column
steps and one row step.  The library's half-sweep kernels rely on exactly
that: each CTA sweeps its tile of one plane with a recomputed 3-column,
1-row halo.  This test runs that schedule (tiles, halo, the two halves in
both directions) in numpy on random symmetric 27-point operators, with small
tiles so that every tile edge and ragged tail occurs, and checks that it
gives the plain 8-colour sweep bit for bit.  It models the schedule, not the
CUDA code: the GPU tests compare the kernels with the oracle."""
import numpy as np
import pytest

OFFS = [(dx, dy, dz) for dz in (-1, 0, 1) for dy in (-1, 0, 1) for dx in (-1, 0, 1)]


def _operator(n, seed):
    """Full 27-entry rows a[k, j, i, o] of a random symmetric operator with
    zero couplings to the boundary, strictly diagonally dominant."""
    rng = np.random.default_rng(seed)
    a = np.zeros((n, n, n, 27))
    inner = lambda v: 1 <= v <= n - 2
    for k in range(1, n - 1):
        for j in range(1, n - 1):
            for i in range(1, n - 1):
                for o, (dx, dy, dz) in enumerate(OFFS):
                    if o >= 13 or not (inner(i + dx) and inner(j + dy) and inner(k + dz)):
                        continue
                    v = -rng.uniform(0.1, 1.0)
                    a[k, j, i, o] = v
                    a[k + dz, j + dy, i + dx, 26 - o] = v
                a[k, j, i, 13] = 30.0 + rng.uniform(0.0, 1.0)
    return a


def _update(a, f, x, i, j, k, xk):
    """Gauss-Seidel update of point (i, j, k); xk(dz) gives the iterate plane
    at k + dz (so a tile's private copies can stand in for the array)."""
    s = 0.0
    for o, (dx, dy, dz) in enumerate(OFFS):
        if o != 13:
            s += a[k, j, i, o] * xk(dz)[j + dy, i + dx]
    return (f[k, j, i] - s) / a[k, j, i, 13]


def _plain_sweep(a, f, x, colours):
    n = x.shape[0]
    for c in colours:
        pi, pj, pk = c & 1, (c >> 1) & 1, c >> 2
        for k in range(2 - pk, n - 1, 2):
            for j in range(2 - pj, n - 1, 2):
                for i in range(2 - pi, n - 1, 2):
                    x[k, j, i] = _update(a, f, x, i, j, k, lambda dz: x[k + dz])


def _half(a, f, xin, xz, xout, parity, forward, ti, tj):
    """One half sweep of all planes of one parity: every tile of ti x tj owned
    points sweeps its region (owned +- 3 columns, +- 1 row) in a private copy
    of the plane, reading the neighbouring planes from xz and writing only
    its owned points to xout."""
    n = xin.shape[0]
    m = n - 2
    order = (0, 1, 2, 3) if forward else (3, 2, 1, 0)
    for k in range(2 - parity, n - 1, 2):
        for j0 in range(1, 1 + m, tj):
            for i0 in range(1, 1 + m, ti):
                plane = xin[k].copy()
                for c in order:
                    pi, pj = c & 1, c >> 1
                    for j in range(j0 - 1, j0 + tj + 1):
                        for i in range(i0 - 3, i0 + ti + 3):
                            if (i & 1) != pi or (j & 1) != pj or not (1 <= i <= m and 1 <= j <= m):
                                continue
                            plane[j, i] = _update(a, f, None, i, j, k,
                                                  lambda dz: plane if dz == 0 else xz[k + dz])
                j1, i1 = min(j0 + tj, m + 1), min(i0 + ti, m + 1)
                xout[k, j0:j1, i0:i1] = plane[j0:j1, i0:i1]


@pytest.mark.parametrize("n,ti,tj", [(11, 4, 2), (17, 6, 4), (17, 10, 6)])
def test_half_sweeps_give_the_eight_colour_sweep(n, ti, tj):
    a = _operator(n, n)
    rng = np.random.default_rng(n + 1)
    f = np.zeros((n, n, n))
    f[1:-1, 1:-1, 1:-1] = rng.uniform(-1, 1, (n - 2,) * 3)
    # down: forward sweep from a zero guess; even planes first (their odd
    # neighbours are still zero), then odd planes against them
    ref = np.zeros((n, n, n))
    _plain_sweep(a, f, ref, range(8))
    x = np.zeros((n, n, n))
    _half(a, f, np.zeros((n, n, n)), np.zeros((n, n, n)), x, 0, True, ti, tj)
    _half(a, f, np.zeros((n, n, n)), x, x, 1, True, ti, tj)
    assert np.array_equal(x, ref)
    # up: reverse sweep from a given iterate; odd planes against the given
    # even planes, then even planes against the finished odd planes
    x0 = np.zeros((n, n, n))
    x0[1:-1, 1:-1, 1:-1] = rng.uniform(-1, 1, (n - 2,) * 3)
    ref = x0.copy()
    _plain_sweep(a, f, ref, range(7, -1, -1))
    y = x0.copy()
    _half(a, f, x0, x0, y, 1, False, ti, tj)
    _half(a, f, x0, y, y, 0, False, ti, tj)
    assert np.array_equal(y, ref)


def test_a_smaller_halo_is_not_enough():
    """With a 2-column halo the forward half misses the three-step colour
    chain x, xy, x at tile edges (the schedule needs 3 columns)."""
    n, ti, tj = 17, 6, 4
    a = _operator(n, 3)
    rng = np.random.default_rng(4)
    f = np.zeros((n, n, n))
    f[1:-1, 1:-1, 1:-1] = rng.uniform(-1, 1, (n - 2,) * 3)
    ref = np.zeros((n, n, n))
    _plain_sweep(a, f, ref, range(8))
    m = n - 2
    x = np.zeros((n, n, n))
    for parity in (0, 1):
        for k in range(2 - parity, n - 1, 2):
            for j0 in range(1, 1 + m, tj):
                for i0 in range(1, 1 + m, ti):
                    plane = np.zeros((n, n))
                    for c in range(4):
                        pi, pj = c & 1, c >> 1
                        for j in range(j0 - 1, j0 + tj + 1):
                            for i in range(i0 - 2, i0 + ti + 2):
                                if (i & 1) != pi or (j & 1) != pj or not (1 <= i <= m and 1 <= j <= m):
                                    continue
                                plane[j, i] = _update(a, f, None, i, j, k, lambda dz: plane if dz == 0 else x[k + dz])
                    j1, i1 = min(j0 + tj, m + 1), min(i0 + ti, m + 1)
                    x[k, j0:j1, i0:i1] = plane[j0:j1, i0:i1]
    assert not np.array_equal(x, ref)
