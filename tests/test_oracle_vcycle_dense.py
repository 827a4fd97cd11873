"""Dense pin of the oracle's degree-1 V(1,1) cycle (Section 3.2).

The oracle runs the V-cycle as a residual-correction program from e = 0.  Here
the same cycle is written as its error-propagation operator, built from closed
forms only (nothing of the oracle's level data is reused):

* level l has m_l elements per axis, n_l = m_l - 1 interior hats, h_l = 1/m_l;
  1D Q1 stiffness (1/h) tridiag(-1, 2, -1) and mass h tridiag(1/6, 2/3, 1/6);
  A_l = K (x) M + M (x) K in 2D, the three-term sum in 3D (Section 2 with p = 1);
* coarsening by 2 while a level has more than 8 elements and an even count, the
  last level solved exactly;
* the 2h -> h embedding S of the hats: weights 1/2, 1, 1/2;
* Gauss-Seidel "red-black" on the 9/27-point stencil read as the parity
  sub-lattices (x_k mod 2 fixed), red ones (even coordinate sum) first, each in
  ascending sub-lattice number; the post-smoother runs the reverse order.  One
  pass over a sub-lattice is prod_{i in c} (I - e_i e_i^T A / a_ii), which equals
  I - D_c A because no two points of a sub-lattice couple (checked here);
* E_l = S_post (I - S B_{l+1} S^T A_l) S_pre, B_L = A_L^{-1},
  B_l = (I - E_l) A_l^{-1}: the V-cycle from zero maps rhs to B_l rhs.

The oracle must reproduce B_0 (2D: the whole matrix, three levels; 3D: three
levels on random right-hand sides) to 1e-12.  A damped or mis-scaled update, a
wrong sub-lattice order, a transposed transfer or a missing post-smoother each
changes B_0 by far more than that.
"""
import numpy as np
import pytest
import scipy.sparse as sp
import scipy.sparse.linalg as spla


def _q1_1d(ml):
    n, h = ml - 1, 1.0 / ml
    e = np.ones(n)
    K = sp.diags([-e[:-1], 2 * e, -e[:-1]], [-1, 0, 1]) / h
    M = sp.diags([e[:-1] / 6, 2 * e / 3, e[:-1] / 6], [-1, 0, 1]) * h
    return sp.csr_matrix(K), sp.csr_matrix(M)


def _op(dim, K, M):
    # x fastest: kron(B_z, kron(B_y, B_x))
    if dim == 2:
        return sp.csr_matrix(sp.kron(M, K) + sp.kron(K, M))
    return sp.csr_matrix(sp.kron(M, sp.kron(M, K)) + sp.kron(M, sp.kron(K, M)) + sp.kron(K, sp.kron(M, M)))


def _embed_1d(mc):
    nc, nf = mc - 1, 2 * mc - 1
    S = sp.lil_matrix((nf, nc))
    for I in range(nc):
        S[2 * I, I] = 0.5
        S[2 * I + 1, I] = 1.0
        S[2 * I + 2, I] = 0.5
    return sp.csr_matrix(S)


def _levels(m0):
    ml = [m0]
    while ml[-1] > 8 and ml[-1] % 2 == 0:
        ml.append(ml[-1] // 2)
    return ml


def _sublattice_order(dim):
    cols = list(range(1 << dim))
    red = [c for c in cols if bin(c).count("1") % 2 == 0]
    black = [c for c in cols if bin(c).count("1") % 2 == 1]
    return red + black


class _DenseVcycle:
    def __init__(self, dim, m0):
        self.dim = dim
        self.ml = _levels(m0)
        self.A, self.S, self.col, self.dinv, self.lu = [], [], [], [], []
        for l, m in enumerate(self.ml):
            K, M = _q1_1d(m)
            A = _op(dim, K, M)
            n = m - 1
            idx = np.arange(n ** dim)
            x = [idx % n, (idx // n) % n] + ([idx // (n * n)] if dim == 3 else [])
            col = sum((xk & 1) << k for k, xk in enumerate(x))
            self.A.append(A)
            self.col.append(col)
            self.dinv.append(1.0 / A.diagonal())
            self.lu.append(spla.splu(sp.csc_matrix(A)))
            if l + 1 < len(self.ml):
                S1 = _embed_1d(self.ml[l + 1])
                S = S1
                for _ in range(dim - 1):
                    S = sp.kron(S1, S)
                self.S.append(sp.csr_matrix(S))
        self.order = _sublattice_order(dim)

    def sublattices_uncoupled(self):
        for A, col in zip(self.A, self.col):
            for c in range(1 << self.dim):
                sel = np.flatnonzero(col == c)
                sub = A[sel][:, sel].tocoo()
                if np.any(sub.row != sub.col):
                    return False
        return True

    def _pass(self, l, c, x):
        w = np.where(self.col[l] == c, self.dinv[l], 0.0)
        return x - (w[:, None] if x.ndim == 2 else w) * (self.A[l] @ x)

    def error_prop(self, l, x):
        """E_l x."""
        for c in self.order:
            x = self._pass(l, c, x)
        A = self.A[l]
        x = x - self.S[l] @ self.approx_inv(l + 1, self.S[l].T @ (A @ x))
        for c in reversed(self.order):
            x = self._pass(l, c, x)
        return x

    def approx_inv(self, l, v):
        """B_l v = (I - E_l) A_l^{-1} v (v: a vector or a matrix of columns)."""
        w = self.lu[l].solve(v)
        if l == len(self.ml) - 1:
            return w
        return w - self.error_prop(l, w)


def test_sublattice_order_is_the_red_black_reading():
    assert _sublattice_order(2) == [0, 3, 1, 2]
    assert _sublattice_order(3) == [0, 3, 5, 6, 1, 2, 4, 7]


def test_vcycle_2d_three_levels_equals_dense_operator(oracle_mod):
    """2D, second level of m = 64 (31^2 DOFs, levels 32 -> 16 -> 8 elements): B_0 in full."""
    P = oracle_mod.Problem(2, 2, 64, sched=oracle_mod.LATTICE, coarse=oracle_mod.VCYCLE)
    D = _DenseVcycle(2, 32)
    assert D.ml == [32, 16, 8] and P.nc == 31
    assert D.sublattices_uncoupled()
    Nc = P.Nc
    B_or = np.empty((Nc, Nc))
    for j in range(Nc):
        e = np.zeros(Nc)
        e[j] = 1.0
        B_or[:, j] = P.coarse_solve(e)
    B_dn = D.approx_inv(0, np.eye(Nc))
    scale = np.abs(B_dn).max()
    assert np.abs(B_or - B_dn).max() <= 1e-12 * scale
    # V(1,1) with reversed post-smoothing is symmetric, and contracts on A_0
    assert np.abs(B_dn - B_dn.T).max() <= 1e-12 * scale
    E = np.eye(Nc) - B_dn @ D.A[0].toarray()
    assert np.abs(np.linalg.eigvals(E)).max() < 0.3


def test_vcycle_3d_three_levels_equals_dense_operator(oracle_mod):
    """3D, second level of m = 64 (31^3 DOFs, levels 32 -> 16 -> 8 elements), random right-hand sides."""
    P = oracle_mod.Problem(3, 2, 64, sched=oracle_mod.LATTICE, coarse=oracle_mod.VCYCLE)
    D = _DenseVcycle(3, 32)
    assert D.ml == [32, 16, 8] and P.nc == 31
    assert D.sublattices_uncoupled()
    rng = np.random.default_rng(20090149)
    for _ in range(3):
        v = rng.uniform(-1.0, 1.0, P.Nc)
        got = P.coarse_solve(v)
        ref = D.approx_inv(0, v)
        assert np.abs(got - ref).max() <= 1e-12 * np.abs(ref).max()


@pytest.mark.parametrize("dim,m0", [(2, 16), (3, 16)])
def test_vcycle_two_levels_equals_dense_operator(oracle_mod, dim, m0):
    """Smaller hierarchies (16 -> 8 elements) on both dimensions."""
    P = oracle_mod.Problem(dim, 3, 2 * m0, sched=oracle_mod.LATTICE, coarse=oracle_mod.VCYCLE)
    D = _DenseVcycle(dim, m0)
    rng = np.random.default_rng(7)
    for _ in range(2):
        v = rng.standard_normal(P.Nc)
        ref = D.approx_inv(0, v)
        assert np.abs(P.coarse_solve(v) - ref).max() <= 1e-12 * np.abs(ref).max()
