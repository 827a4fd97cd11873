"""Pins for the oracle's operator, schedules and multiplicative Schwarz step
(Section 3.1.1).

Independent references: the explicit Kronecker matrix (numpy), a brute-force
coupling check of every colour class, and the paper's product formula
prod_j (I - V_j^T A_j^{-1} V_j A) for the error propagation, built densely
with numpy on tiny grids.
"""
import itertools

import numpy as np
import pytest


def _dense_A(oracle_mod, dim, p, m):
    K, M = oracle_mod.assemble_1d(p, m)
    if dim == 2:
        return np.kron(K, M) + np.kron(M, K), K, M
    return (np.kron(K, np.kron(M, M)) + np.kron(M, np.kron(K, M))
            + np.kron(M, np.kron(M, K))), K, M


def _block(dim, n, c, r):
    """Grid indices of the s^d box around centre index c, clipped, x fastest."""
    cz, cy, cx = (c // (n * n), (c // n) % n, c % n) if dim == 3 else (0, c // n, c % n)
    out = []
    zr = range(cz - r, cz + r + 1) if dim == 3 else [0]
    for z in zr:
        for y in range(cy - r, cy + r + 1):
            for x in range(cx - r, cx + r + 1):
                if 0 <= x < n and 0 <= y < n and 0 <= z < (n if dim == 3 else 1):
                    out.append(x + n * (y + n * z))
    return np.array(out)


@pytest.mark.parametrize("dim,p,m", [(2, 2, 5), (2, 5, 4), (3, 2, 4), (3, 3, 3)])
def test_apply_A_matches_kronecker(oracle_mod, dim, p, m):
    A, K, M = _dense_A(oracle_mod, dim, p, m)
    u = np.random.default_rng(0).standard_normal(A.shape[0])
    assert np.allclose(oracle_mod.apply_A(dim, K, M, u, p), A @ u, atol=1e-12)


SCHED_CASES = [
    # dim, p, m, kind, tile, period, stride
    (2, 2, 14, 1, 0, 5, 2),
    (2, 3, 14, 1, 0, 7, 2),
    (2, 4, 12, 2, 7, 7, 2),
    (2, 2, 20, 2, 5, 5, 2),
    (2, 5, 15, 2, 10, 10, 3),
    # the tile sides the GPU kernels compile (20 for p = 2, 5; 21 for p = 3, 4; 22 for p = 6), with
    # at least two tiles of one phase
    (2, 2, 44, 2, 20, 5, 2),
    (2, 3, 45, 2, 21, 7, 2),
    (2, 4, 44, 2, 21, 7, 2),
    (2, 5, 45, 2, 20, 10, 3),
    (2, 6, 44, 2, 22, 11, 4),
    # the default LATTICE colourings of the 7x7 blocks (p = 7, 8)
    (2, 7, 44, 1, 0, 14, 5),
    (2, 8, 50, 1, 0, 17, 4),
    (3, 2, 8, 1, 0, 5, 2),
    (3, 3, 9, 2, 7, 7, 2),
    (3, 2, 12, 2, 5, 5, 2),   # 3D tile side = period, two tiles of one phase per axis
]


@pytest.mark.parametrize("dim,p,m,kind,tile,period,stride", SCHED_CASES)
def test_schedule_colours_are_coupling_free(oracle_mod, dim, p, m, kind, tile, period, stride):
    """Within a colour no block shares a DOF with, or reads a DOF written by, another."""
    A, _, _ = _dense_A(oracle_mod, dim, p, m)
    n = m + p - 2
    s = oracle_mod.block_size(p)
    r = (s - 1) // 2
    colour, order, ncol = oracle_mod.schedule(dim, n, s, p, kind, tile, period, stride)
    nz = A != 0
    assert sorted(order.tolist()) == list(range(n ** dim))
    assert np.all(np.diff(colour[order]) >= 0)
    for col in np.unique(colour):
        cent = np.nonzero(colour == col)[0]
        blocks = [_block(dim, n, c, r) for c in cent]
        reads = [np.nonzero(nz[b].any(axis=0))[0] for b in blocks]
        for a, b in itertools.combinations(range(len(cent)), 2):
            assert not np.intersect1d(blocks[a], blocks[b]).size
            assert not np.intersect1d(blocks[a], reads[b]).size
            assert not np.intersect1d(blocks[b], reads[a]).size


def test_schedule_rejects_short_period(oracle_mod):
    with pytest.raises(ValueError):
        oracle_mod.schedule(2, 20, 3, 2, 1, 0, 4, 1)  # q < s + p
    with pytest.raises(ValueError):
        oracle_mod.schedule(2, 20, 3, 2, 1, 0, 6, 2)  # gcd(g, q) != 1
    with pytest.raises(ValueError):
        oracle_mod.schedule(2, 20, 3, 2, 2, 4, 5, 2)  # tile < q


@pytest.mark.parametrize("dim,p,m,kind,tile", [(2, 2, 6, 0, 0), (2, 2, 8, 1, 0), (2, 3, 9, 2, 7),
                                               (2, 5, 5, 1, 0), (2, 6, 6, 1, 0), (2, 7, 6, 1, 0),
                                               (2, 8, 6, 0, 0), (3, 2, 4, 1, 0), (3, 3, 3, 0, 0)])
def test_schwarz_matches_product_formula(oracle_mod, dim, p, m, kind, tile):
    """u_new - u* = prod_j (I - V_j^T A_j^{-1} V_j A) (u - u*), blocks in schedule order."""
    A, K, M = _dense_A(oracle_mod, dim, p, m)
    n = m + p - 2
    N = n ** dim
    s = oracle_mod.block_size(p)
    r = (s - 1) // 2
    _, order, _ = oracle_mod.schedule(dim, n, s, p, kind, tile)
    rng = np.random.default_rng(11)
    b = rng.standard_normal(N)
    u = rng.standard_normal(N)
    ustar = np.linalg.solve(A, b)
    E = np.eye(N)
    for c in order:
        B = _block(dim, n, c, r)
        V = np.zeros((len(B), N))
        V[np.arange(len(B)), B] = 1.0
        E = (np.eye(N) - V.T @ np.linalg.solve(V @ A @ V.T, V @ A)) @ E
    got = oracle_mod.schwarz_sweep(dim, K, M, p, s, order, b, u)
    ref = ustar + E @ (u - ustar)
    assert np.allclose(got, ref, atol=1e-11 * np.abs(ref).max())


def test_order_within_colour_is_irrelevant(oracle_mod):
    dim, p, m = 2, 3, 24
    n = m + p - 2
    s = 3
    K, M = oracle_mod.assemble_1d(p, m)
    colour, order, _ = oracle_mod.schedule(dim, n, s, p, 1)
    rng = np.random.default_rng(3)
    b = rng.standard_normal(n * n)
    u = rng.standard_normal(n * n)
    # reverse the order inside every colour class
    perm = np.lexsort((-order, colour[order]))
    order2 = order[perm].astype(np.int32)
    assert not np.array_equal(order, order2)
    a1 = oracle_mod.schwarz_sweep(dim, K, M, p, s, order, b, u)
    a2 = oracle_mod.schwarz_sweep(dim, K, M, p, s, order2, b, u)
    assert np.array_equal(a1, a2)


def test_block_size_table(oracle_mod):
    import json, os
    gold = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "paper_tables.json")))
    for p, s in gold["block_size"].items():
        if p.startswith("_"):
            continue
        assert oracle_mod.block_size(int(p)) == s


@pytest.mark.parametrize("p,tile", [(3, 7), (4, 7)])
def test_tile3d_phases_are_coupling_free_at_size(oracle_mod, p, tile):
    """The 3D TILE sides the GPU compiles (7 for p = 3, 4) on a grid with several tiles of
    one phase per axis (29-31 DOFs per axis; the dense check above is too large here):
    within a colour, any two clipped blocks are more than p apart along some axis, so
    neither shares a DOF with nor reads a DOF of the other (A couples DOFs at most p apart
    per axis, the 1D bands having half-width p)."""
    m = 28
    n = m + p - 2
    s = oracle_mod.block_size(p)
    r = (s - 1) // 2
    colour, order, ncol = oracle_mod.schedule(3, n, s, p, 2, tile, 7, 2)
    assert sorted(order.tolist()) == list(range(n ** 3))
    idx = np.arange(n ** 3)
    cx, cy, cz = idx % n, (idx // n) % n, idx // (n * n)
    lo = np.stack([np.maximum(c - r, 0) for c in (cx, cy, cz)], axis=1)
    hi = np.stack([np.minimum(c + r, n - 1) for c in (cx, cy, cz)], axis=1)
    for col in np.unique(colour):
        cent = np.nonzero(colour == col)[0]
        a_lo, a_hi = lo[cent], hi[cent]
        # pairwise: separated by more than p along at least one axis
        sep = (a_lo[:, None, :] > a_hi[None, :, :] + p) | (a_lo[None, :, :] > a_hi[:, None, :] + p)
        ok = sep.any(axis=2)
        np.fill_diagonal(ok, True)
        assert ok.all(), (col, cent[np.argwhere(~ok)[0]])


@pytest.mark.parametrize("dim,p,m,tile,period,stride,groups", [
    (2, 6, 44, 22, 11, 4, 4),     # the grouped TILE order of degree 6 (4 colour groups)
    (2, 2, 40, 10, 5, 2, 3),
    (2, 4, 44, 21, 7, 2, 2),
])
def test_grouped_tile_colours_are_coupling_free(oracle_mod, dim, p, m, tile, period, stride, groups):
    """Every colour of the grouped TILE order is one parallel phase (no shared or read DOF)."""
    A, _, _ = _dense_A(oracle_mod, dim, p, m)
    n = m + p - 2
    s = oracle_mod.block_size(p)
    r = (s - 1) // 2
    colour, order, ncol = oracle_mod.schedule(dim, n, s, p, 2, tile, period, stride, groups)
    nz = A != 0
    assert sorted(order.tolist()) == list(range(n ** dim))
    for col in np.unique(colour):
        cent = np.nonzero(colour == col)[0]
        blocks = [_block(dim, n, c, r) for c in cent]
        reads = [np.nonzero(nz[b].any(axis=0))[0] for b in blocks]
        for a, b in itertools.combinations(range(len(cent)), 2):
            assert not np.intersect1d(blocks[a], blocks[b]).size
            assert not np.intersect1d(blocks[a], reads[b]).size
            assert not np.intersect1d(blocks[b], reads[a]).size


@pytest.mark.parametrize("p,n,tile,q,g", [(2, 40, 10, 5, 2), (6, 70, 22, 11, 4), (4, 45, 21, 7, 2)])
def test_grouped_tile_order_limits_and_definition(oracle_mod, p, n, tile, q, g):
    """groups = 1 is the TILE order and groups = q^2 the LATTICE order; in between, the
    order is (colour group, tile phase, lattice colour, index) written out here directly:
    centre (x, y) has tile phase (x // T) % 2 + 2 ((y // T) % 2), lattice colour l =
    rank(x mod q) + q rank(y mod q) with rank(o) = o g^-1 mod q (tile sides are multiples
    of q), and group floor(l groups / q^2)."""
    s = oracle_mod.block_size(p)
    _, o_tile, _ = oracle_mod.schedule(2, n, s, p, 2, tile, q, g)
    _, o_g1, _ = oracle_mod.schedule(2, n, s, p, 2, tile, q, g, 1)
    assert np.array_equal(o_tile, o_g1)
    _, o_lat, _ = oracle_mod.schedule(2, n, s, p, 1, 0, q, g)
    _, o_gq, _ = oracle_mod.schedule(2, n, s, p, 2, tile, q, g, q * q)
    # both orders visit the lattice colours in the same sequence; inside a colour the
    # LATTICE order is by index, the grouped one by tile phase then index
    rank = {o: (o * pow(g, -1, q)) % q for o in range(q)}
    lat = lambda c: rank[(c % n) % q] + q * rank[(c // n) % q]
    assert [lat(c) for c in o_gq] == [lat(c) for c in o_lat]
    for groups in (2, 3, q):
        _, o, _ = oracle_mod.schedule(2, n, s, p, 2, tile, q, g, groups)
        key = []
        for c in range(n * n):
            x, y = c % n, c // n
            l = lat(c)
            tp = (x // tile) % 2 + 2 * ((y // tile) % 2)
            key.append((l * groups // (q * q), tp, l, c))
        want = [k[3] for k in sorted(key)]
        assert o.tolist() == want, groups
