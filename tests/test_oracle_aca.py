"""Pins for the oracle's three-way ACA (Algorithm 1), its face ACA and
recompression, eq. (norm), and the compressed apply (eq. (product))."""
import numpy as np
import pytest

from inputs import workloads
from oracle import aca3, apply as A, freqs, quadrature as Q, tree


def _rand(rng, *shape):
    return rng.standard_normal(shape) + 1j * rng.standard_normal(shape)


def test_aca2_exact_on_rank_r_matrix():
    rng = np.random.default_rng(0)
    for r in (1, 3, 7):
        X = _rand(rng, 40, r) @ _rand(rng, r, 33)
        U, V = aca2_dense(X, 1e-12)
        assert U.shape[1] <= r + 1
        assert np.linalg.norm(X - U @ V.conj().T) < 1e-12 * np.linalg.norm(X)


def aca2_dense(X, eps):
    return aca3.aca2(lambda i: X[i, :], lambda j: X[:, j], X.shape[0], X.shape[1], eps)


def test_aca2_smooth_kernel_tolerance_and_interpolation():
    x = np.linspace(0, 1, 60)
    y = np.linspace(3, 4, 50)
    X = 1.0 / np.abs(x[:, None] - y[None, :]) * np.exp(-(0.5 + 2j) * np.abs(x[:, None] - y[None, :]))
    for eps in (1e-4, 1e-8):
        U, V = aca2_dense(X, eps)
        err = np.linalg.norm(X - U @ V.conj().T) / np.linalg.norm(X)
        assert err < 10 * eps
    # ACA interpolates the selected crosses: rows i_t / columns j_t are exact
    U, V = aca2_dense(X, 1e-6)
    S = U @ V.conj().T
    res = np.abs(X - S)
    assert np.sum(res.max(axis=1) < 1e-12 * np.abs(X).max()) >= U.shape[1]


def test_aca2_zero_rows_are_skipped_and_zero_matrix_gives_rank0():
    X = np.zeros((10, 8), dtype=complex)
    U, V = aca2_dense(X, 1e-6)
    assert U.shape == (10, 0)
    X[7, 3] = 2.0 + 1.0j
    U, V = aca2_dense(X, 1e-6)
    assert U.shape[1] == 1 and np.allclose(U @ V.conj().T, X)


def test_recompress_preserves_product_and_truncates():
    rng = np.random.default_rng(1)
    U = _rand(rng, 30, 6)
    V = _rand(rng, 25, 6)
    U2, V2 = aca3.recompress(U, V, 1e-14)
    assert np.linalg.norm(U @ V.conj().T - U2 @ V2.conj().T) < 1e-12 * np.linalg.norm(U @ V.conj().T)
    assert np.allclose(V2.conj().T @ V2, np.eye(V2.shape[1]), atol=1e-12)
    # a rank-2 product written with 6 columns recompresses to rank 2
    U = _rand(rng, 30, 2) @ _rand(rng, 2, 6)
    U2, V2 = aca3.recompress(U, V, 1e-10)
    assert U2.shape[1] == 2


def test_aca3_rank1_separable_exact():
    rng = np.random.default_rng(2)
    op = aca3.SeparableBlock(_rand(rng, 1, 20), _rand(rng, 1, 17), _rand(rng, 1, 9))
    res = aca3.aca3(op, 1e-6)
    assert res.rank == 1
    D = op.dense()
    assert np.linalg.norm(D - res.dense(20, 17, 9)) < 1e-13 * np.linalg.norm(D)


@pytest.mark.parametrize("R", [2, 3, 5])
def test_aca3_rank_r_separable_recovered(R):
    rng = np.random.default_rng(10 + R)
    # decaying weights keep the cross pivots well separated
    c = _rand(rng, R, 12) * (0.3 ** np.arange(R))[:, None]
    op = aca3.SeparableBlock(_rand(rng, R, 22), _rand(rng, R, 19), c)
    res = aca3.aca3(op, 1e-10)
    assert res.rank <= R
    D = op.dense()
    assert np.linalg.norm(D - res.dense(22, 19, 12)) < 1e-9 * np.linalg.norm(D)


def _bem_block(name="cube768", kernel="slp", pick="largest"):
    """The largest admissible block of a workload (or block `pick`)."""
    w = workloads.get(name)
    g = Q.Geometry(w.verts, w.tris)
    T = tree.build(w.verts, w.tris, w.leaf, w.eta)
    fs = freqs.frequency_set(w.freq)
    s_u = fs["s"][fs["uniq"]]
    far = [b for b in range(T.blocks.shape[0]) if T.blocks[b, 4] == 1]
    sizes = [(T.blocks[b, 1] - T.blocks[b, 0]) * (T.blocks[b, 3] - T.blocks[b, 2]) for b in far]
    b = far[int(np.argmax(sizes))] if pick == "largest" else far[pick]
    rb, re, cb, ce, _ = T.blocks[b]
    ef = lambda I, J, s: Q.entries(g, kernel, I, J, s)
    op = aca3.BemBlock(ef, T.perm[rb:re], T.perm[cb:ce], s_u)
    D = Q.dense(g, kernel, s_u, rows=T.perm[rb:re], cols=T.perm[cb:ce])
    return op, D, s_u


@pytest.mark.parametrize("dense_max", [aca3.DENSE_MAX, -1])
def test_aca3_bem_block_tolerance_norm_recursion_and_fiber_interpolation(dense_max):
    op, D, s_u = _bem_block()
    eps3 = 1e-4
    res = aca3.aca3(op, eps3, s_abs=np.abs(s_u), dense_max=dense_max)
    M, N, Ku = D.shape
    C = res.dense(M, N, Ku)
    assert res.rank >= 2
    # brute force: the approximant meets the tolerance on the whole block
    assert np.linalg.norm(D - C) <= 10 * eps3 * np.linalg.norm(D)
    # eq. (norm): the recursive norm equals the dense norm of the approximant
    assert abs(res.norm2_history[res.rank - 1] - np.linalg.norm(C) ** 2) < 1e-10 * np.linalg.norm(C) ** 2
    # the fiber at the last kept pivot is reproduced exactly
    last = res.crosses[-1]
    assert np.max(np.abs(C[last.i, last.j, :] - D[last.i, last.j, :])) < 1e-10 * np.abs(D).max()
    # the face at each used frequency is reproduced to the face tolerance
    for c in res.crosses:
        assert np.linalg.norm(C[:, :, c.k] - D[:, :, c.k]) < 1e-4 * np.linalg.norm(D[:, :, c.k])
    # the first frequency is always the first one used
    assert res.crosses[0].k == 0


def test_aca3_dlp_zero_block_has_rank0():
    """Double-layer blocks whose collocation points all lie in the planes of
    the column elements vanish identically; they are detected as zero blocks
    after testing further frequencies, and other blocks are not."""
    w = workloads.get("lshape3072")
    g = Q.Geometry(w.verts, w.tris)
    T = tree.build(w.verts, w.tris, w.leaf, w.eta)
    fs = freqs.frequency_set(w.freq)
    s_u = fs["s"][fs["uniq"]]
    ef = lambda I, J, s: Q.entries(g, "dlp", I, J, s)
    zero, nonzero = 0, 0
    for b in range(T.blocks.shape[0]):
        rb, re, cb, ce, adm = T.blocks[b]
        if not adm:
            continue
        R, Cc = T.perm[rb:re], T.perm[cb:ce]
        d = np.einsum("ijd,jd->ij", g.centroid[R][:, None, :] - g.v0[Cc][None, :, :], g.normal[Cc])
        is_zero = bool(np.all(d == 0.0))
        if (is_zero and zero < 3) or (not is_zero and nonzero < 2):
            res = aca3.aca3(aca3.BemBlock(ef, R, Cc, s_u), 1e-4, s_abs=np.abs(s_u))
            assert (res.rank == 0) == is_zero and res.zero_block == is_zero
            zero += is_zero
            nonzero += not is_zero
        if zero == 3 and nonzero == 2:
            break
    assert zero == 3 and nonzero == 2


@pytest.mark.parametrize("dense_max", [aca3.DENSE_MAX, -1])
def test_compressed_apply_matches_dense_apply(dense_max):
    w = workloads.get("cube768")
    g = Q.Geometry(w.verts, w.tris)
    T = tree.build(w.verts, w.tris, 32, 1.0)
    fs = freqs.frequency_set(workloads.bdf2_spec(8, 0.1))
    s_all, uniq, partner = fs["s"], fs["uniq"], fs["partner"]
    s_u = s_all[uniq]
    ef = lambda I, J, s: Q.entries(g, "slp", I, J, s)
    res = {}
    for b, (rb, re, cb, ce, adm) in enumerate(T.blocks):
        if adm:
            res[b] = aca3.aca3(aca3.BemBlock(ef, T.perm[rb:re], T.perm[cb:ce], s_u), 1e-4,
                               s_abs=np.abs(s_u), dense_max=dense_max)
    assert len(res) > 0
    W = workloads.densities(w.E, 8, 3)
    yc = A.compressed_apply(T, res, ef, s_all, uniq, partner, W)
    yd = A.dense_apply(ef, w.E, s_all, W)
    assert np.linalg.norm(yc - yd) <= 10 * 1e-4 * np.linalg.norm(yd)
    # the far-field part alone also meets the tolerance
    far_only = A.compressed_apply(T, res, lambda I, J, s: np.zeros((I.size, s.size), complex),
                                  s_all, uniq, partner, W)
    yfar = np.zeros(w.E, dtype=complex)
    for b, (rb, re, cb, ce, adm) in enumerate(T.blocks):
        if adm:
            R, Cc = T.perm[rb:re], T.perm[cb:ce]
            D = Q.dense(g, "slp", s_all, rows=R, cols=Cc)
            yfar[R] += np.einsum("ijk,jk->i", D, W[Cc, :])
    assert np.linalg.norm(far_only - yfar) <= 10 * 1e-4 * np.linalg.norm(yfar)


def test_expand_fibers_uses_conjugate_partners():
    K = 8
    uniq, partner = freqs.bdf2_unique(K)
    f = np.arange(1, uniq.size + 1) * (1 + 1j)
    a, b = A.expand_fibers(f, uniq, partner, K)
    assert np.allclose(a[uniq], f)
    for u, k in enumerate(uniq):
        if partner[k] != k:
            assert b[partner[k]] == np.conj(f[u])
    assert np.all(a[[k for k in range(K) if k not in uniq]] == 0)


def test_dense_faces_rank_r_exact_and_match_algorithm1():
    """Small blocks use the exact residual face (Algorithm 1 as written):
    rank-R separable tensors are recovered in R crosses, and every face of the
    approximant at a used frequency equals the data there."""
    rng = np.random.default_rng(21)
    R = 3
    c = _rand(rng, R, 10) * (0.2 ** np.arange(R))[:, None]
    op = aca3.SeparableBlock(_rand(rng, R, 12), _rand(rng, R, 9), c)
    res = aca3.aca3(op, 1e-12)             # 12 x 9 <= DENSE_MAX: dense faces
    assert res.rank <= R
    D = op.dense()
    C = res.dense(12, 9, 10)
    assert np.linalg.norm(D - C) < 1e-12 * np.linalg.norm(D)
    for x in res.crosses:
        assert np.max(np.abs(C[:, :, x.k] - D[:, :, x.k])) < 1e-12 * np.abs(D).max()
    # forcing low-rank faces reaches the same tensor
    res2 = aca3.aca3(aca3.SeparableBlock(op.a, op.b, op.c), 1e-12, dense_max=-1)
    assert np.linalg.norm(D - res2.dense(12, 9, 10)) < 1e-10 * np.linalg.norm(D)


def test_dense_faces_bem_block_tolerance():
    op, D, s_u = _bem_block("lshape768")
    assert op.M * op.N <= aca3.DENSE_MAX
    res = aca3.aca3(op, 1e-4, s_abs=np.abs(s_u))
    C = res.dense(*D.shape)
    assert np.linalg.norm(D - C) <= 10 * 1e-4 * np.linalg.norm(D)
    # each face at a used frequency is reproduced up to the later crosses' contribution there
    assert res.crosses[0].k == 0 and res.crosses[0].U.shape == (op.M, op.N)


def test_confirmed_stop_fixes_two_plane_dlp_block():
    """A double-layer block of the L-shape whose rows and columns each span
    the x = 0 and z = 1 faces ([[0, X], [Y, 0]] coplanarity): partial-pivot
    face ACA never visits Y and the block ends with ~47 % error (reproduced
    with sample_check=False); with the sampled confirmation of face
    convergence and of the stop the block meets the tolerance."""
    w = workloads.get("lshape12288")
    g = Q.Geometry(w.verts, w.tris)
    T = tree.build(w.verts, w.tris, w.leaf, w.eta)
    fs = freqs.frequency_set(w.freq)
    s_u = fs["s"][fs["uniq"]]
    far = np.nonzero(T.blocks[:, 4] == 1)[0]
    rb, re, cb, ce, _ = T.blocks[far[3660]]
    R, C = T.perm[rb:re], T.perm[cb:ce]
    assert {tuple(n) for n in g.normal[R]} == {(-1.0, 0.0, 0.0), (0.0, 0.0, 1.0)}
    ef = lambda I, J, s: Q.entries(g, "dlp", I, J, s)
    D = Q.dense(g, "dlp", s_u, rows=R, cols=C)
    lit = aca3.aca3(aca3.BemBlock(ef, R, C, s_u), 1e-4, s_abs=np.abs(s_u), sample_check=False)
    assert np.linalg.norm(lit.dense(*D.shape) - D) > 0.1 * np.linalg.norm(D)
    res = aca3.aca3(aca3.BemBlock(ef, R, C, s_u), 1e-4, s_abs=np.abs(s_u))
    assert np.linalg.norm(res.dense(*D.shape) - D) <= 10 * 1e-4 * np.linalg.norm(D)
    # the faces now also cover the Y part: larger face ranks
    assert sum(c.face_rank for c in res.crosses) > sum(c.face_rank for c in lit.crosses)


def test_sample_positions_cover_the_block():
    pos = aca3.sample_entries(96, 96)
    assert len(set(pos)) == 32
    assert len({i for i, _ in pos}) == 32 and len({j for _, j in pos}) == 32
    assert all(0 <= i < 7 and 0 <= j < 5 for i, j in aca3.sample_entries(7, 5))


# ---------------------------------------------------------------- next frequency and the literal stop

def _staircase_tensor(scale3: float = 1.0):
    """Rank-3 tensor sum_t a_t (x) b_t (x) c_t whose three terms live on
    disjoint column ranges (columns 3t..3t+2 of a 12 x 9 block; the a_t are
    dense, so every row of a face meets every term; Ku = 10) and whose fibers
    are built so that Algorithm 1's frequency sequence follows from the
    definitions alone (the fiber at a pivot in column range t is term t's):

      c_0: c_0[0] = 1 (the only term at k = 0), largest other entry at k = 3
           (0.9), second largest at k = 5 (0.8);
      c_1: c_1[0] = 0, c_1[3] = 1 (the only term left at k = 3), largest
           entry off {0, 3} at k = 7 (0.7), small at k = 5;
      c_2: c_2[0] = c_2[3] = 0, c_2[7] = scale3 (the only term left at k = 7).

    Face 1 (k = 0) is term 0 alone, so f_1 = c_0 / c_0[0] and C^(1) is term 0
    exactly; the argmax over unused k of |f_1| is k = 3 (k = 0 itself has
    |f_1| = 1 > 0.9 and must be excluded).  Face 2 (k = 3) is term 1 alone,
    f_2 = c_1 / c_1[3], next k = 7 (taking |f_1| instead of |f_2| would give
    k = 5).  Face 3 (k = 7) is term 2 alone and C^(3) equals the tensor."""
    rng = np.random.default_rng(77)
    M, N, Ku = 12, 9, 10
    a = np.zeros((3, M), complex)
    b = np.zeros((3, N), complex)
    for t in range(3):
        a[t] = _rand(rng, M)
        b[t, 3 * t:3 * t + 3] = _rand(rng, 3)

    def fiber(mags):
        return np.asarray(mags) * np.exp(2j * np.pi * rng.random(Ku))

    c = np.zeros((3, Ku), complex)
    c[0] = fiber([1.0, 0.3, 0.2, 0.9, 0.4, 0.8, 0.1, 0.35, 0.25, 0.15])
    c[0, 0] = 1.0
    c[1] = fiber([0.0, 0.2, 0.3, 1.0, 0.25, 0.05, 0.4, 0.7, 0.1, 0.45])
    c[2] = fiber([0.0, 0.5, 0.3, 0.0, 0.2, 0.4, 0.1, 1.0, 0.45, 0.35]) * scale3
    return a, b, c


@pytest.mark.parametrize("dense_max", [aca3.DENSE_MAX, -1])
@pytest.mark.parametrize("sample_check", [True, False])
def test_next_frequency_rule_sequence(dense_max, sample_check):
    """Algorithm 1's k_{l+1} = argmax over unused k of |f_l[k]| on a tensor
    whose frequency sequence is known in advance (0, 3, 7)."""
    a, b, c = _staircase_tensor()
    op = aca3.SeparableBlock(a, b, c)
    res = aca3.aca3(op, 1e-4, dense_max=dense_max, sample_check=sample_check)
    assert [x.k for x in res.crosses] == [0, 3, 7]
    # each cross carries one term: its pivot lies in that term's column range
    for t, x in enumerate(res.crosses):
        assert 3 * t <= x.j < 3 * t + 3
        assert np.allclose(x.f, c[t] / c[t, x.k], rtol=0, atol=1e-13)
    D = op.dense()
    assert np.linalg.norm(D - res.dense(12, 9, 10)) < 1e-13 * np.linalg.norm(D)
    # a fourth face is zero up to rounding: it is either detected as zero or
    # computed from rounding noise and dropped by the stopping test
    assert res.rank == 3 and res.computed in (3, 4)


@pytest.mark.parametrize("dense_max", [aca3.DENSE_MAX, -1])
def test_literal_stop_drops_the_last_cross(dense_max):
    """Algorithm 1 as written: the cross that meets the stopping test is
    computed and discarded (r = l - 1).  With the third term at 1e-6 of the
    others, cross 3 meets ||H_3|| ||f_3|| <= eps3 ||C^(3)|| for eps3 = 1e-4;
    the returned approximant is terms 0 and 1, off by exactly the third term."""
    a, b, c = _staircase_tensor(scale3=1e-6)
    op = aca3.SeparableBlock(a, b, c)
    D = op.dense()
    third = np.einsum("i,j,k->ijk", a[2], b[2], c[2])
    for sample_check in (False, True):
        res = aca3.aca3(aca3.SeparableBlock(a, b, c), 1e-4, dense_max=dense_max, sample_check=sample_check)
        assert res.computed == 3 and res.rank == 2 == res.computed - 1
        assert [x.k for x in res.crosses] == [0, 3]
        R = D - res.dense(12, 9, 10)
        assert np.linalg.norm(R - third) < 1e-13 * np.linalg.norm(D)
        assert np.linalg.norm(R) <= 1e-4 * np.linalg.norm(D)


def test_literal_stop_bem_block_meets_tolerance():
    """On the largest single-layer block of the cube the literal test is
    valid: rank = crosses computed - 1 and the approximant meets the
    tolerance against the dense block."""
    op, D, s_u = _bem_block()
    eps3 = 1e-4
    res = aca3.aca3(op, eps3, s_abs=np.abs(s_u), dense_max=-1, sample_check=False)
    assert res.rank == res.computed - 1 and res.rank >= 2
    C = res.dense(*D.shape)
    assert np.linalg.norm(D - C) <= 10 * eps3 * np.linalg.norm(D)


def test_perfreq_dense_apply_terms():
    """Y[:, l] = A(s_l) w_l: each column is the dense matrix at s_l times w_l,
    and the columns sum to the SUM-mode apply of eq. (product)."""
    w = workloads.get("cube48")
    g = Q.Geometry(w.verts, w.tris)
    s_all = freqs.bdf2(6, 0.1, (1e-8) ** (1.0 / 12))
    W = workloads.densities(w.E, 6, 5)
    ef = lambda I, J, s: Q.entries(g, "slp", I, J, s)
    Y = A.dense_apply_perfreq(ef, w.E, s_all, W)
    D = Q.dense(g, "slp", s_all)
    for l in range(6):
        assert np.allclose(Y[:, l], D[:, :, l] @ W[:, l], rtol=1e-13, atol=0)
    y = A.dense_apply(ef, w.E, s_all, W)
    assert np.allclose(Y.sum(axis=1), y, rtol=1e-13, atol=0)


# ---------------------------------------------------------------- the pivot estimate of eq. (index)

def test_index_pivot_is_exact_on_rank1_faces():
    """For a rank-1 face u v^H the estimate of eq. (index) returns
    (argmax |u|, argmax |v|), which is the largest entry of the face."""
    rng = np.random.default_rng(41)
    for _ in range(5):
        u = _rand(rng, 23, 1)
        v = _rand(rng, 17, 1)
        H = u @ v.conj().T
        i, j = aca3.index_pivot(u, v)
        assert (i, j) == np.unravel_index(np.argmax(np.abs(H)), H.shape)
        assert i == int(np.argmax(np.abs(u))) and j == int(np.argmax(np.abs(v)))


def test_index_pivot_matches_eq_index_on_recompressed_faces():
    """On recompressed factors (U = U' Sigma, V orthonormal) the row is eq.
    (index)'s argmax_i sum_k |u_ik sigma_k|, the column the largest entry of
    that row; the pivot is within sqrt(r N) of the face's largest entry
    (|H_ij| >= ||H_i,:|| / sqrt(N) = ||U_i,:|| / sqrt(N) >= sum_k |U_ik| / sqrt(r N))."""
    rng = np.random.default_rng(42)
    U0, V0 = _rand(rng, 30, 4), _rand(rng, 26, 4)
    U, V = aca3.recompress(U0, V0, 1e-14)
    assert np.allclose(V.conj().T @ V, np.eye(V.shape[1]))
    i, j = aca3.index_pivot(U, V)
    assert i == int(np.argmax(np.abs(U).sum(axis=1)))
    H = U @ V.conj().T
    assert j == int(np.argmax(np.abs(H[i])))
    r, N = U.shape[1], V.shape[0]
    assert np.abs(H[i, j]) >= np.abs(U[i]).sum() / np.sqrt(r * N)
    assert np.abs(H[i, j]) >= np.abs(H).max() / np.sqrt(r * N)


def test_index_pivot_avoids_vanishing_entry_on_block_diagonal_face():
    """A face [[A, 0], [0, B]] with A 2 x 4 (entries ~1.5) and B 8 x 4
    (entries ~1): the largest row bound lies in A's rows (1.5 * 2 > 1 * 2) and
    the largest column bound in B's columns (sqrt(8) > 1.5 sqrt(2)); their
    common entry is zero, so the column is taken in the selected row."""
    rng = np.random.default_rng(43)
    U = np.zeros((10, 2), complex)
    V = np.zeros((8, 2), complex)
    U[:2, 0] = 1.5 * (1 + _rand(rng, 2) * 0.01)       # rows of A
    V[:4, 0] = 1.0 * (1 + _rand(rng, 4) * 0.01)       # columns of A
    U[2:, 1] = 1.0 * (1 + _rand(rng, 8) * 0.01)       # rows of B
    V[4:, 1] = 1.0 * (1 + _rand(rng, 4) * 0.01)       # columns of B
    i, j = aca3.index_pivot(U, V)
    H = U @ V.conj().T
    assert i < 2 and j < 4 and abs(H[i, j]) > 0
    # the independent column bound would have picked a column of B: H[i, j'] = 0
    cu = np.linalg.norm(U, axis=0)
    jb = int(np.argmax(np.abs(V) @ cu))
    assert jb >= 4 and H[i, jb] == 0


def test_index_pivot_single_layer_block_meets_tolerance():
    """Algorithm 1 with the pivot of eq. (index) on the largest single-layer
    block of the cube (the paper reports the estimate works for the single
    layer) meets the tolerance against the dense block."""
    op, D, s_u = _bem_block()
    eps3 = 1e-4
    res = aca3.aca3(op, eps3, s_abs=np.abs(s_u), dense_max=-1, pivot="index")
    C = res.dense(*D.shape)
    assert np.linalg.norm(D - C) <= 10 * eps3 * np.linalg.norm(D)


# ---------------------------------------------------------------- 3D-ACA on the H-matrix as a whole

def test_whole_matrix_rank_is_set_by_all_blocks():
    """Two blocks, each a rank-1 separable tensor: per block the ACA needs one
    cross each; on the matrix as a whole the fibers are shared, so two
    blocks with different frequency dependence need two crosses (the
    combined tensor has rank 2), and one when they share it."""
    rng = np.random.default_rng(51)
    a1, b1, a2, b2 = _rand(rng, 1, 12), _rand(rng, 1, 10), _rand(rng, 1, 9), _rand(rng, 1, 11)
    c1, c2 = _rand(rng, 1, 8), _rand(rng, 1, 8)
    for ca, cb, want in ((c1, c2, 2), (c1, 0.5 * c1, 1)):
        ops = [aca3.SeparableBlock(a1, b1, ca), aca3.SeparableBlock(a2, b2, cb)]
        res = aca3.aca3_whole(ops, 1e-8)
        assert res.rank == want
        for b, (op, M, N) in enumerate(((ops[0], 12, 10), (ops[1], 9, 11))):
            D = op.dense()
            assert np.linalg.norm(res.dense(b, M, N, 8) - D) <= 1e-12 * np.linalg.norm(D)
        per_block = [aca3.aca3(aca3.SeparableBlock(a1, b1, ca), 1e-8).rank,
                     aca3.aca3(aca3.SeparableBlock(a2, b2, cb), 1e-8).rank]
        assert per_block == [1, 1] and res.rank >= max(per_block)


def test_whole_matrix_norm_is_the_sum_of_block_norms():
    """eq. (norm) evaluated per block and summed: the recursive norm equals
    the Frobenius norm of all blocks' approximants together."""
    rng = np.random.default_rng(52)
    R = 3
    ops = [aca3.SeparableBlock(_rand(rng, R, 14), _rand(rng, R, 12), _rand(rng, R, 9) * (0.3 ** np.arange(R))[:, None]),
           aca3.SeparableBlock(_rand(rng, R, 10), _rand(rng, R, 13), _rand(rng, R, 9) * (0.3 ** np.arange(R))[:, None])]
    res = aca3.aca3_whole(ops, 1e-10)
    tot = sum(np.linalg.norm(res.dense(b, op.M, op.N, 9)) ** 2 for b, op in enumerate(ops))
    assert abs(res.norm2_history[res.rank - 1] - tot) <= 1e-10 * tot
    # the shared fiber is exact at its pivot entry (cross interpolation)
    b, i, j, k = res.pivots[-1]
    D = ops[b].dense()
    C = res.dense(b, ops[b].M, ops[b].N, 9)
    assert np.max(np.abs(C[i, j, :] - D[i, j, :])) <= 1e-10 * np.abs(D).max()


def test_whole_matrix_bem_blocks_meet_tolerance():
    """Eight admissible single-layer blocks of the cube compressed as one
    H-matrix meet the tolerance on all blocks together, with a rank no
    smaller than the largest per-block rank."""
    w = workloads.get("cube768")
    g = Q.Geometry(w.verts, w.tris)
    T = tree.build(w.verts, w.tris, w.leaf, w.eta)
    fs = freqs.frequency_set(w.freq)
    s_u = fs["s"][fs["uniq"]]
    ef = lambda I, J, s: Q.entries(g, "slp", I, J, s)
    far = [b for b in range(T.blocks.shape[0]) if T.blocks[b, 4] == 1]
    rng = np.random.default_rng(53)
    pick = rng.choice(len(far), 8, replace=False)
    ops, Ds = [], []
    for p in pick:
        rb, re, cb, ce, _ = T.blocks[far[p]]
        ops.append(aca3.BemBlock(ef, T.perm[rb:re], T.perm[cb:ce], s_u))
        Ds.append(Q.dense(g, "slp", s_u, rows=T.perm[rb:re], cols=T.perm[cb:ce]))
    res = aca3.aca3_whole(ops, 1e-4, s_abs=np.abs(s_u))
    err = sum(np.linalg.norm(res.dense(b, *D.shape) - D) ** 2 for b, D in enumerate(Ds)) ** 0.5
    ref = sum(np.linalg.norm(D) ** 2 for D in Ds) ** 0.5
    assert err <= 10 * 1e-4 * ref
    per_block = [aca3.aca3(aca3.BemBlock(ef, op.rows, op.cols, s_u), 1e-4, s_abs=np.abs(s_u), dense_max=-1,
                           sample_check=False).rank for op in ops]
    assert res.rank >= max(per_block)
