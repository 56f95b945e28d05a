"""Oracle: the three-way (generalised) ACA of one admissible block.

TEST INFRASTRUCTURE ONLY (see oracle/__init__.py).

Follows Algorithm 1 ("3D ACA") of the paper, with the implementation
remarks of the same section, in complex128:

  l = 0, k_1 = first frequency, C^(0) = 0
  repeat
    l += 1
    face:   H_l ~ ENTRY(:, :, k_l) - C^(l-1)[:, :, k_l], approximated by
            partial-pivot ACA (the faces are compressed with ACA, tolerance
            eps_face = eps3 / 100, "eps = 100 eps_ACA") and recompressed by
            QR of both factors + SVD of R_U R_V^H (first remark)
    pivot:  (i_l, j_l) = argmax |H_l[i, j]| over the dense expansion of the
            low-rank face (last remark: "expanding to the dense block"), or
            optionally the cheaper estimate of eq. (index) from the
            recompressed factors
    fiber:  f_l[k] = (ENTRY(i_l, j_l, k) - C^(l-1)[i_l, j_l, k]) / H_l[i_l, j_l]
    norm:   ||C^(l)||_F^2 by eq. (norm), i.e. the double sum over
            <H_d, H_d'>_F <f_d, f_d'>, accumulated over the new terms
    stop when ||H_l||_F ||f_l||_2 <= eps3 ||C^(l)||_F ; the rank is l - 1
    (the last cross is dropped, as in Algorithm 1), or when every frequency
    is used (rank l)
    k_{l+1} = argmax over not-yet-used k of |f_l[k]|

Readings where the paper is silent (all shared with the CUDA path):

* The tensor is the block restricted to the unique frequencies (one of each
  conjugate pair, Appendix A: only half of the frequencies need to be
  computed); k_1 = 0 (every block starts with the first frequency).
* argmax ties: smallest index (row-major for (i, j)).  k_{l+1} excludes
  frequencies already used (|f_l[k_l]| = 1 would otherwise repeat k_l).
* Face ACA (Bebendorf's partial pivoting): start with the block's first row;
  column pivot j = argmax |residual row|; next row = argmax over unused rows
  of |u|; a row whose residual is exactly zero is marked used and the
  smallest unused row is tried next; stop when ||u|| ||v|| <= eps_face ||S||_F
  (||S||_F updated recursively), or at min(M, N) or `max_face_rank` crosses.
* Recompression truncates singular values sigma_i < eps_face * sigma_1.
* A zero face (no row with a nonzero residual) at k_l: the paper only says
  that some frequencies are tested to confirm a zero block.  Up to three more
  unused frequencies are tested (the last unique one, the middle one, the one
  of largest |s|); if all faces are zero the block ends with rank l - 1.
* Dense faces for small blocks: the paper also runs the three-way ACA
  without low-rank approximation in the faces ("No Lwr", Section 5.1).  For
  a block with M N <= dense_max the face H_l is the exact residual face
  ENTRY(:, :, k_l) - C^(l-1)[:, :, k_l] (Algorithm 1 as written) and the
  pivot is its largest entry; such blocks are where a face of rank r at the
  face tolerance has r (M + N) >= M N, i.e. the low-rank form is no smaller
  than the dense one.  A zero face then means an exactly zero residual face.
* Confirmed stop (sample_check): the stopping test only measures the newest
  cross.  On double-layer blocks whose rows and columns span two planar
  faces (entries zero between coplanar elements, [[0, X], [Y, 0]]), the
  pivots stay in the dominant part and the test passes at a frequency where
  the approximation is already exact while other frequencies are off by
  40-50 %.  When the test passes, the residual of the approximant including
  the newest cross is therefore evaluated at S = 32 fixed sample entries
  (rows (2s+1) M // 64, columns (2 (11 s mod 32) + 1) N // 64) over all
  frequencies; if its Frobenius norm exceeds eps3 times that of the sampled
  data, the newest cross is kept and the next frequency is the unused one
  with the largest sampled residual.
* Confirmed face convergence (sample_check): partial pivoting misses a
  [[0, X], [Y, 0]] face (every visited row and column stays in X).  When the
  face ACA's test passes, its residual is evaluated at the same 32 sample
  positions; if (M N / 32) sum |R_s|^2 > eps_face^2 ||S||_F^2 the ACA
  continues from the row of the largest sampled residual.
"""
from __future__ import annotations

import numpy as np


class BlockEntries:
    """ENTRY restricted to one block and the unique frequencies (abstract)."""

    M: int
    N: int
    Ku: int

    def row(self, i: int, k: int) -> np.ndarray:
        raise NotImplementedError

    def col(self, j: int, k: int) -> np.ndarray:
        raise NotImplementedError

    def fiber(self, i: int, j: int) -> np.ndarray:
        raise NotImplementedError

    def face(self, k: int) -> np.ndarray:
        raise NotImplementedError


class BemBlock(BlockEntries):
    """Collocation entries of a block (rows/cols are ORIGINAL element ids)."""

    def __init__(self, entry_fn, rows: np.ndarray, cols: np.ndarray, s_u: np.ndarray):
        self.f = entry_fn            # f(I, J, s) -> [n, nk]
        self.rows = np.asarray(rows)
        self.cols = np.asarray(cols)
        self.s = np.asarray(s_u)
        self.M, self.N, self.Ku = self.rows.size, self.cols.size, self.s.size
        self.generated = 0

    def row(self, i, k):
        self.generated += self.N
        return self.f(np.full(self.N, self.rows[i]), self.cols, self.s[k:k + 1])[:, 0]

    def col(self, j, k):
        self.generated += self.M
        return self.f(self.rows, np.full(self.M, self.cols[j]), self.s[k:k + 1])[:, 0]

    def fiber(self, i, j):
        self.generated += self.Ku
        return self.f(self.rows[i:i + 1], self.cols[j:j + 1], self.s)[0]

    def face(self, k):
        self.generated += self.M * self.N
        I = np.repeat(self.rows, self.N)
        J = np.tile(self.cols, self.M)
        return self.f(I, J, self.s[k:k + 1])[:, 0].reshape(self.M, self.N)


class SeparableBlock(BlockEntries):
    """Synthetic test tensor A[i, j, k] = sum_t a[t, i] b[t, j] c[t, k]."""

    def __init__(self, a: np.ndarray, b: np.ndarray, c: np.ndarray):
        self.a, self.b, self.c = (np.asarray(x, dtype=np.complex128) for x in (a, b, c))
        self.M, self.N, self.Ku = self.a.shape[1], self.b.shape[1], self.c.shape[1]
        self.generated = 0

    def row(self, i, k):
        self.generated += self.N
        return (self.a[:, i] * self.c[:, k]) @ self.b

    def col(self, j, k):
        self.generated += self.M
        return (self.b[:, j] * self.c[:, k]) @ self.a

    def fiber(self, i, j):
        self.generated += self.Ku
        return (self.a[:, i] * self.b[:, j]) @ self.c

    def face(self, k):
        self.generated += self.M * self.N
        return np.einsum("ti,tj,t->ij", self.a, self.b, self.c[:, k])

    def dense(self) -> np.ndarray:
        return np.einsum("ti,tj,tk->ijk", self.a, self.b, self.c)


SAMPLES = 32


def sample_entries(M: int, N: int) -> list[tuple[int, int]]:
    """The fixed residual-check positions of an M x N block."""
    return [((2 * s + 1) * M // (2 * SAMPLES), (2 * ((11 * s) % SAMPLES) + 1) * N // (2 * SAMPLES))
            for s in range(SAMPLES)]


def aca2(row_fn, col_fn, M: int, N: int, eps: float, max_rank: int | None = None,
         sample_check: bool = False):
    """Partial-pivot ACA of a matrix given by residual row/column callbacks.

    Returns U [M, r], V [N, r] with the approximant S = U V^H.
    """
    cap = min(M, N) if max_rank is None else min(M, N, max_rank)
    us: list[np.ndarray] = []
    vs: list[np.ndarray] = []
    used = np.zeros(M, dtype=bool)
    norm2 = 0.0
    i = 0
    while len(us) < cap:
        while True:
            row = row_fn(i).astype(np.complex128)
            for u_t, v_t in zip(us, vs):
                row = row - u_t[i] * np.conj(v_t)
            used[i] = True
            mag = row.real * row.real + row.imag * row.imag
            j = int(np.argmax(mag))
            if mag[j] > 0.0:
                break
            free = np.nonzero(~used)[0]
            if free.size == 0:
                return _stack(us, M), _stack(vs, N)
            i = int(free[0])
        delta = row[j]
        v = np.conj(row / delta)
        u = col_fn(j).astype(np.complex128)
        for u_t, v_t in zip(us, vs):
            u = u - u_t * np.conj(v_t[j])
        cross = 0.0
        for u_t, v_t in zip(us, vs):
            cross += 2.0 * (np.vdot(u_t, u) * np.vdot(v, v_t)).real
        nu2 = float(np.vdot(u, u).real)
        nv2 = float(np.vdot(v, v).real)
        norm2 += cross + nu2 * nv2
        us.append(u)
        vs.append(v)
        if np.sqrt(nu2 * nv2) <= eps * np.sqrt(norm2):
            if not sample_check:
                break
            pos = sample_entries(M, N)
            res = np.array([row_fn(a)[b] - sum(u_t[a] * np.conj(v_t[b]) for u_t, v_t in zip(us, vs))
                            for a, b in pos])
            mres = res.real * res.real + res.imag * res.imag
            if (M * N / SAMPLES) * mres.sum() <= eps * eps * norm2:
                break
            i = pos[int(np.argmax(mres))][0]
            continue
        free = np.nonzero(~used)[0]
        if free.size == 0:
            break
        mag = u.real * u.real + u.imag * u.imag
        i = int(free[int(np.argmax(mag[free]))])
    return _stack(us, M), _stack(vs, N)


def _stack(cols: list[np.ndarray], n: int) -> np.ndarray:
    if not cols:
        return np.zeros((n, 0), dtype=np.complex128)
    return np.stack(cols, axis=1)


def recompress(U: np.ndarray, V: np.ndarray, eps: float):
    """U V^H = Q_U (R_U R_V^H) Q_V^H, SVD of the core, truncation at
    sigma_i < eps sigma_1.  Returns (U' = Q_U X Sigma, V' = Q_V Y)."""
    if U.shape[1] == 0:
        return U, V
    Qu, Ru = np.linalg.qr(U)
    Qv, Rv = np.linalg.qr(V)
    X, sig, Yh = np.linalg.svd(Ru @ Rv.conj().T)
    r = int(np.count_nonzero(sig >= eps * sig[0]))
    return Qu @ (X[:, :r] * sig[:r]), Qv @ Yh[:r].conj().T


class Cross:
    __slots__ = ("U", "V", "f", "i", "j", "k")

    def __init__(self, U, V, f, i, j, k):
        self.U, self.V, self.f, self.i, self.j, self.k = U, V, f, i, j, k

    @property
    def face_rank(self) -> int:
        return self.U.shape[1]


class Result:
    def __init__(self, crosses, computed, norm2_history, zero_block):
        self.crosses: list[Cross] = crosses
        self.computed = computed           # crosses computed incl. the dropped one
        self.norm2_history = norm2_history # ||C^(l)||_F^2 after each cross (eq. (norm))
        self.zero_block = zero_block

    @property
    def rank(self) -> int:
        return len(self.crosses)

    def dense(self, M: int, N: int, Ku: int) -> np.ndarray:
        out = np.zeros((M, N, Ku), dtype=np.complex128)
        for c in self.crosses:
            out += (c.U @ c.V.conj().T)[:, :, None] * c.f[None, None, :]
        return out


DENSE_MAX = 48 * 48


def index_pivot(U: np.ndarray, V: np.ndarray) -> tuple[int, int]:
    """Pivot estimate of eq. (index) (Section 4, last implementation remark)
    for a recompressed face U V^H with orthonormal columns in V and U = (u_k
    sigma_k): the row i = argmax_i sum_k |u_ik sigma_k| bounds the entries of
    row i.  Written for any factor pair as i = argmax_i sum_k |U_ik| ||V_:k||
    (the same numbers when V has orthonormal columns).  The column is then
    found "the analogous way" in that row: j = argmax_j |(U V^H)[i, j]|, the
    largest entry of the selected row (O(N r), like the row estimate's
    O(M r)); ties -> smallest index.  (Choosing j by the independent column
    bound sum_k ||U_:k|| |V_jk| can pair a large row with a large column whose
    common entry vanishes, e.g. on block-diagonal faces, and the fiber
    division then blows up.)"""
    cv = np.linalg.norm(V, axis=0)
    i = int(np.argmax(np.abs(U) @ cv))
    row = U[i, :] @ V.conj().T
    j = int(np.argmax(row.real * row.real + row.imag * row.imag))
    return i, j


def aca3(op: BlockEntries, eps3: float, eps_face: float | None = None,
         s_abs: np.ndarray | None = None, max_face_rank: int | None = None,
         k1: int = 0, dense_max: int = DENSE_MAX, sample_check: bool = True,
         pivot: str = "dense") -> Result:
    """Algorithm 1 on one block (see module docstring for the readings).
    Blocks with M N <= dense_max use exact dense faces (dense_max < 0: never);
    sample_check confirms each stop on fixed sample entries.  pivot = "dense":
    the largest entry of the face's dense expansion (the variant of all the
    paper's results); "index": the estimate of eq. (index) on low-rank faces
    (dense faces keep their exact largest entry)."""
    if eps_face is None:
        eps_face = eps3 / 100.0
    M, N, Ku = op.M, op.N, op.Ku
    crosses: list[Cross] = []
    faces: list[np.ndarray] = []       # dense H_d, for eq. (norm)
    used = np.zeros(Ku, dtype=bool)
    norm2 = 0.0
    hist: list[float] = []
    k = k1
    ell = 0

    dense = M * N <= dense_max

    def face_at(kk: int):
        if dense:
            H = op.face(kk)
            for c in crosses:
                H = H - c.f[kk] * (c.U @ c.V.conj().T)
            if not np.any(H != 0):
                return np.zeros((M, 0), complex), np.zeros((N, 0), complex)
            return H, np.eye(N, dtype=complex)

        def row_fn(i):
            r = op.row(i, kk)
            for c in crosses:
                r = r - c.f[kk] * (c.U[i, :] @ c.V.conj().T)
            return r

        def col_fn(j):
            cc = op.col(j, kk)
            for c in crosses:
                cc = cc - c.f[kk] * (c.U @ c.V[j, :].conj())
            return cc

        return aca2(row_fn, col_fn, M, N, eps_face, max_face_rank, sample_check=sample_check)

    while True:
        ell += 1
        U, V = face_at(k)
        used[k] = True
        if U.shape[1] == 0:
            cands = []
            for kk in (Ku - 1, Ku // 2,
                       int(np.argmax(s_abs)) if s_abs is not None else Ku - 1):
                if not used[kk] and kk not in cands:
                    cands.append(kk)
            found = False
            for kk in cands[:3]:
                used[kk] = True
                U, V = face_at(kk)
                if U.shape[1] > 0:
                    k = kk
                    found = True
                    break
            if not found:
                return Result(crosses, ell - 1, hist, zero_block=(ell == 1))
        if not dense:
            U, V = recompress(U, V, eps_face)
        H = U @ V.conj().T
        if pivot == "index" and not dense:
            ip, jp = index_pivot(U, V)
        else:
            mag = H.real * H.real + H.imag * H.imag
            flat = int(np.argmax(mag))
            ip, jp = divmod(flat, N)
        fib = op.fiber(ip, jp)
        for c, Hd in zip(crosses, faces):
            fib = fib - Hd[ip, jp] * c.f
        f = fib / H[ip, jp]
        # eq. (norm): add the terms of the double sum that involve cross l
        new = 0.0
        for c, Hd in zip(crosses, faces):
            new += 2.0 * (np.vdot(Hd, H) * np.vdot(c.f, f)).real
        nH2 = float(np.vdot(H, H).real)
        nf2 = float(np.vdot(f, f).real)
        norm2 += new + nH2 * nf2
        hist.append(norm2)
        cross = Cross(U, V, f, ip, jp, k)
        resid = None
        if np.sqrt(nH2 * nf2) <= eps3 * np.sqrt(norm2):
            if not sample_check or used.all():
                return Result(crosses, ell, hist, zero_block=False)
            A_s = np.array([op.fiber(i, j) for i, j in sample_entries(M, N)])          # [S, Ku]
            C_s = np.zeros_like(A_s)
            for c, Hd in zip(crosses + [cross], faces + [H]):
                C_s += np.array([Hd[i, j] for i, j in sample_entries(M, N)])[:, None] * c.f[None, :]
            R_s = A_s - C_s
            if np.linalg.norm(R_s) <= eps3 * np.linalg.norm(A_s):
                return Result(crosses, ell, hist, zero_block=False)
            resid = np.sum(R_s.real ** 2 + R_s.imag ** 2, axis=0)
        crosses.append(cross)
        faces.append(H)
        if ell == Ku or used.all():
            return Result(crosses, ell, hist, zero_block=False)
        fm = f.real * f.real + f.imag * f.imag if resid is None else resid
        fm = np.where(used, -1.0, fm)
        k = int(np.argmax(fm))


class WholeResult:
    """Three-way ACA of several blocks as one H-matrix: per block the faces
    H_p^b = U_p^b (V_p^b)^H, and one fiber f_p shared by all blocks."""

    def __init__(self, faces, fibers, pivots, computed, norm2_history):
        self.faces = faces                 # faces[b][p] = (U, V)
        self.fibers = fibers               # fibers[p] = f_p  [Ku]
        self.pivots = pivots               # pivots[p] = (block, i, j, k)
        self.computed = computed
        self.norm2_history = norm2_history

    @property
    def rank(self) -> int:
        return len(self.fibers)

    def dense(self, b: int, M: int, N: int, Ku: int) -> np.ndarray:
        out = np.zeros((M, N, Ku), dtype=np.complex128)
        for (U, V), f in zip(self.faces[b], self.fibers):
            out += (U @ V.conj().T)[:, :, None] * f[None, None, :]
        return out


def aca3_whole(ops: list, eps3: float, eps_face: float | None = None, s_abs: np.ndarray | None = None,
               max_face_rank: int | None = None, k1: int = 0) -> WholeResult:
    """The other choice of Section 4's first implementation remark: the
    three-way ACA applied to the H-matrix as a whole.  The tensor is the
    admissible part of the matrix over the (unique) frequencies; a face is
    the H-matrix at k_l (every block's residual face compressed by ACA and
    recompressed, as in `aca3`), the pivot is the largest entry of that face
    over all blocks, and one fiber per cross serves every block:

      H_l^b ~ ENTRY_b(:, :, k_l) - sum_{p<l} f_p[k_l] H_p^b
      (b*, i, j) = argmax_b,i,j |H_l^b[i, j]|
      f_l[k] = (ENTRY_b*(i, j, k) - sum_{p<l} H_p^b*[i, j] f_p[k]) / H_l^b*[i, j]
      ||C^(l)||^2 = sum_b (eq. (norm) of block b)       ("evaluated for each
                                                           block and summed up")
      stop when ||H_l||_F ||f_l||_2 <= eps3 ||C^(l)||_F (||H_l||^2 = sum_b ||H_l^b||^2),
      rank l - 1 as in Algorithm 1; k_{l+1} = argmax over unused k of |f_l[k]|.

    A face that is zero in every block triggers the same extra frequency
    tests as `aca3`.  The literal stopping test (no sampled confirmation)."""
    if eps_face is None:
        eps_face = eps3 / 100.0
    nb = len(ops)
    Ku = ops[0].Ku
    faces: list[list] = [[] for _ in range(nb)]
    dense_faces: list[list] = [[] for _ in range(nb)]
    fibers: list[np.ndarray] = []
    pivots: list[tuple] = []
    used = np.zeros(Ku, dtype=bool)
    norm2 = 0.0
    hist: list[float] = []
    k = k1
    ell = 0

    def block_face(b: int, kk: int):
        op = ops[b]

        def row_fn(i):
            r = op.row(i, kk)
            for (U, V), f in zip(faces[b], fibers):
                r = r - f[kk] * (U[i, :] @ V.conj().T)
            return r

        def col_fn(j):
            c = op.col(j, kk)
            for (U, V), f in zip(faces[b], fibers):
                c = c - f[kk] * (U @ V[j, :].conj())
            return c

        U, V = aca2(row_fn, col_fn, op.M, op.N, eps_face, max_face_rank)
        return recompress(U, V, eps_face)

    while True:
        ell += 1
        cand = [k] + [kk for kk in (Ku - 1, Ku // 2, int(np.argmax(s_abs)) if s_abs is not None else Ku - 1)]
        new = None
        for c_i, kk in enumerate(cand):
            if c_i > 0 and (used[kk] or kk in cand[:c_i]):
                continue
            used[kk] = True
            fl = [block_face(b, kk) for b in range(nb)]
            if any(U.shape[1] > 0 for U, _ in fl):
                new, k = fl, kk
                break
            if c_i == 0 and len(fibers) == 0:
                pass
        if new is None:
            return WholeResult(faces, fibers, pivots, ell - 1, hist)
        Hs = [U @ V.conj().T for U, V in new]
        best, bp = -1.0, None
        for b, H in enumerate(Hs):
            mag = H.real * H.real + H.imag * H.imag
            m = int(np.argmax(mag))
            if mag.flat[m] > best:
                best, bp = float(mag.flat[m]), (b, *divmod(m, ops[b].N))
        b, ip, jp = bp
        fib = ops[b].fiber(ip, jp)
        for Hd, f in zip(dense_faces[b], fibers):
            fib = fib - Hd[ip, jp] * f
        f = fib / Hs[b][ip, jp]
        add = 0.0
        nH2 = 0.0
        for bb in range(nb):
            for Hd, fd in zip(dense_faces[bb], fibers):
                add += 2.0 * (np.vdot(Hd, Hs[bb]) * np.vdot(fd, f)).real
            nH2 += float(np.vdot(Hs[bb], Hs[bb]).real)
        nf2 = float(np.vdot(f, f).real)
        norm2 += add + nH2 * nf2
        hist.append(norm2)
        if np.sqrt(nH2 * nf2) <= eps3 * np.sqrt(norm2):
            return WholeResult(faces, fibers, pivots, ell, hist)
        for bb in range(nb):
            faces[bb].append(new[bb])
            dense_faces[bb].append(Hs[bb])
        fibers.append(f)
        pivots.append((b, ip, jp, k))
        if used.all():
            return WholeResult(faces, fibers, pivots, ell, hist)
        fm = np.where(used, -1.0, f.real * f.real + f.imag * f.imag)
        k = int(np.argmax(fm))
