"""Plain, slow FP64 CPU oracle for the bilayer product-quantization search path.

TEST INFRASTRUCTURE ONLY.  This module exists to check the CUDA library against
the paper.  Only ``tests/``, ``__graft_entry__.smoke()`` and ``bench.py`` (its
CPU-baseline leg and its ``--impl reference`` arm) may import it.  The library
package ``paper_1404_1831_gb300`` never imports, links or calls anything here,
and nothing here imports the library: the two share no code.  Inputs come from
``synthdata`` (the seeded generator module, which holds none of the method's
arithmetic).

Every function follows the step of Babenko & Lempitsky, "Improving Bilayer
Product Quantization for Billion-Scale Approximate Nearest Neighbors in High
Dimensions" (arXiv:1404.1831) that its docstring names.  Arithmetic is FP64 for
distances and exact integer (int64 / Python int) for k-means means.

Readings of points the paper leaves open:
  * Codebooks live on the integer grid: every k-means update rounds the mean
    half up to an integer, floor((2*sum + n) / (2*n)).  Points are integers in
    [0, 255], so every distance in this module is an exact integer below 2^53 and
    the FP64 results below are exact whatever the summation order.
  * K-means starts from the first K training vectors (HBPQ local codebooks start
    from the global residual codebook of the same sub-quantizer); an empty
    cluster keeps its previous centroid; assignment ties go to the lowest index.
  * Cells are ordered by (d1[i] + d2[j], cell id i*T + j); a query visits whole
    cells until the visited cells hold at least L points (the shortest such
    prefix).  Points inside a cell are stored in ascending point id.
  * Final ranking is by (distance, id); fewer than k candidates pad with id -1
    and distance +inf.  The true nearest neighbour breaks ties by lowest id.

Parity pins (tests/test_oracle_*.py) tie each function to something other than
itself: brute force on tiny inputs, hand-checkable k-means cases, codebook
training on learn sets whose coarse centroids and residual codebooks are written
out by hand (global and local), the multi-sequence heap against the full-sort
definition, hand-computed reconstructions (Eq. 7 and §3.2), the FBPQ
decomposition and the HBPQ table regrouping against explicit reconstruction, the
zero-quantization special case against brute-force k-NN, and the paper's printed
memory sizes.
"""

from __future__ import annotations

import dataclasses
import heapq

import numpy as np

KSUB = 256  # codewords per PQ codebook (§2.1, §2.3.1: one byte per index)

# ----------------------------------------------------------------------------
# Squared distances and nearest codewords
# ----------------------------------------------------------------------------


def sq_dists(X, C):
    """All squared Euclidean distances ||x - c||^2, shape (len(X), len(C)), FP64.

    Written as ||x||^2 - 2<x, c> + ||c||^2 with a library matmul as one step.
    For integer-valued inputs every term is an integer below 2^53, so the result
    equals the plain sum of squared differences exactly (pinned in the tests).
    """
    X = np.asarray(X, dtype=np.float64)
    C = np.asarray(C, dtype=np.float64)
    return (X * X).sum(1)[:, None] - 2.0 * (X @ C.T) + (C * C).sum(1)[None, :]


def nearest(X, C, chunk=8192):
    """Index of the nearest codeword for each row of X; ties go to the lowest index.

    This is the vector quantizer of §2.1 and the coarse quantizers q^1, q^2 of
    Eqs. 2-3 (argmin over the codebook).  np.argmin returns the first minimum.
    """
    X = np.asarray(X)
    out = np.empty(len(X), dtype=np.int64)
    for s in range(0, len(X), chunk):
        out[s:s + chunk] = np.argmin(sq_dists(X[s:s + chunk], C), axis=1)
    return out


# ----------------------------------------------------------------------------
# K-means (Lloyd) on the integer grid — §2.3.1 and §3.2 (Eq. 11)
# ----------------------------------------------------------------------------


def rounded_mean(sums, counts):
    """Mean rounded half up to an integer: floor((2*sum + n) / (2*n)), exact in int64."""
    sums = np.asarray(sums, dtype=np.int64)
    counts = np.asarray(counts, dtype=np.int64)
    return (2 * sums + counts[:, None]) // (2 * counts[:, None])


def kmeans(X, K, iters, init=None):
    """Lloyd's K-means as used for every codebook of §2.3.1 (and §3.2 locally).

    X: (n, d) integer-valued.  init: (K, d) starting centroids, default the first
    K rows of X.  Each iteration assigns every point to its nearest centroid (ties
    to the lowest index), then moves each non-empty centroid to the rounded mean
    of its points; an empty cluster keeps its centroid.
    Returns (centroids int64 (K, d), distortion after each assignment step).
    """
    X = np.asarray(X, dtype=np.int64)
    if init is None:
        if len(X) < K:
            raise ValueError("need at least K training vectors")
        C = X[:K].copy()
    else:
        C = np.asarray(init, dtype=np.int64).copy()
    history = []
    for _ in range(iters):
        a = nearest(X, C)
        diff = X - C[a]
        history.append(int((diff * diff).sum()))
        counts = np.bincount(a, minlength=K)
        sums = np.zeros_like(C)
        np.add.at(sums, a, X)
        nz = counts > 0
        C[nz] = rounded_mean(sums[nz], counts[nz])
    return C, history


# ----------------------------------------------------------------------------
# Codebooks: Multi-D-ADC (§2.3.1) and HBPQ local codebooks (§3.2)
# ----------------------------------------------------------------------------


@dataclasses.dataclass
class Codebooks:
    D: int
    T: int
    M: int
    C1: np.ndarray            # (T, D/2) first-half coarse codebook C^1
    C2: np.ndarray            # (T, D/2) second-half coarse codebook C^2
    R: np.ndarray             # (M, 256, D/M) global residual codebooks R_1..R_M
    Q: np.ndarray | None = None  # (T, M/2, 256, D/M) HBPQ local codebooks Q^i_k
    S: np.ndarray | None = None  # (T, M/2, 256, D/M) HBPQ local codebooks S^j_k
    # OPQ ("optimized" variants, §2.3 / §3.2): orthogonal rotations, FP64.  rot0 (D, D)
    # acts on the vectors before the coarse quantization; rot1, rot2 (D/2, D/2) act on
    # the two halves of the displacement before the residual PQ.  None: no rotation.
    rot0: np.ndarray | None = None
    rot1: np.ndarray | None = None
    rot2: np.ndarray | None = None

    @property
    def sub(self):
        return self.D // self.M

    @property
    def rotated(self):
        return self.rot0 is not None

    def coarse_space(self, X):
        """x' = rot0 x (the space of the coarse codebooks C^1, C^2)."""
        X = np.asarray(X)
        return X @ self.rot0.T if self.rotated else X

    def residual_space(self, V):
        """[rot1 v^1; rot2 v^2] for vectors of the coarse space (the space of R_k)."""
        V = np.asarray(V)
        if not self.rotated:
            return V
        h = self.D // 2
        return np.concatenate([V[..., :h] @ self.rot1.T, V[..., h:] @ self.rot2.T], axis=-1)

    def residual_centroids(self):
        """The coarse centroids in the residual space, [rot1 c^1_i], [rot2 c^2_j]."""
        if not self.rotated:
            return self.C1, self.C2
        return (np.asarray(self.C1, np.float64) @ self.rot1.T, np.asarray(self.C2, np.float64) @ self.rot2.T)


def check_shape(D, T, M):
    """The PQ split must align with the two halves (Eq. 9 sums k <= M/2 against c^1)."""
    if D % 2 or M % 2 or (D // 2) % (M // 2):
        raise ValueError("need D even, M even and D/M dividing D/2")


def coarse_cells(X, C1, C2):
    """Cell (i, j) of each point: i = q^1(x^1), j = q^2(x^2) (Eqs. 2-4)."""
    h = C1.shape[1]
    return nearest(X[:, :h], C1), nearest(X[:, h:], C2)


def train_multi_d_adc(learn, T, M, iters):
    """Codebooks of §2.3.1: C^1, C^2 by K-means on the halves, then R_1..R_M by
    K-means on the displacements of all learn points from their cell centroids
    (the set written under Eq. 4)."""
    learn = np.asarray(learn, dtype=np.int64)
    D = learn.shape[1]
    check_shape(D, T, M)
    h, s = D // 2, D // M
    C1, _ = kmeans(learn[:, :h], T, iters)
    C2, _ = kmeans(learn[:, h:], T, iters)
    i, j = coarse_cells(learn, C1, C2)
    disp = learn - np.concatenate([C1[i], C2[j]], axis=1)
    R = np.stack([kmeans(disp[:, k * s:(k + 1) * s], KSUB, iters)[0] for k in range(M)])
    return Codebooks(D=D, T=T, M=M, C1=C1, C2=C2, R=R)


def round_half_up(V):
    """Nearest integer, halves up: floor(v + 1/2) (the integer-grid reading)."""
    return np.floor(np.asarray(V, np.float64) + 0.5).astype(np.int64)


def allocate_eigenvalues(lam, groups):
    """Eigenvalue allocation of parametric OPQ (Ge et al., "Optimized Product
    Quantization", 2013): eigenvalues in descending order (ties by index) are dealt
    to `groups` subspaces of len(lam)/groups dimensions each; each goes to the
    non-full subspace with the smallest sum of log eigenvalues so far (ties to the
    lower subspace), which balances the products of the subspaces' variances.
    Returns, per subspace, the eigenvalue indices in the order they were dealt."""
    lam = np.asarray(lam, np.float64)
    d = len(lam)
    cap = d // groups
    order = sorted(range(d), key=lambda i: (-lam[i], i))
    buckets = [[] for _ in range(groups)]
    logsum = [0.0] * groups
    for i in order:
        b = min((g for g in range(groups) if len(buckets[g]) < cap), key=lambda g: (logsum[g], g))
        buckets[b].append(i)
        logsum[b] += float(np.log(max(lam[i], 1e-12)))
    return buckets


def opq_rotation(X, groups):
    """Parametric OPQ rotation for `groups` subspaces: the eigenvectors of the
    covariance of X (FP64), arranged by allocate_eigenvalues so that subspace g
    holds rows g*d/groups .. (g+1)*d/groups - 1.  Each eigenvector's largest-magnitude
    component is made positive (first such index on ties)."""
    X = np.asarray(X, np.float64)
    mu = X.mean(0)
    C = (X.T @ X) / len(X) - np.outer(mu, mu)
    lam, V = np.linalg.eigh(C)
    rows = []
    for b in allocate_eigenvalues(lam, groups):
        for i in b:
            v = V[:, i]
            if v[int(np.argmax(np.abs(v)))] < 0:
                v = -v
            rows.append(v)
    return np.stack(rows)


def train_opq(learn, T, M, iters, rotations=None):
    """OMulti-D-OADC codebooks (§2.3, the optimized Multi-D-ADC of the paper's
    experiments; the learner is the parametric OPQ solution): rot0 from the learn set
    for the two halves, coarse codebooks on the rotated learn set, then rot1, rot2 from
    the two halves of the displacements for M/2 subspaces each, and R_k on the rotated
    displacements.  Reading (integer grid): the rotated learn vectors and the rotated
    displacements are rounded half up before K-means, so every codebook is integral
    in its (rotated) space.  rotations: (rot0, rot1, rot2) to use instead of learning."""
    learn = np.asarray(learn, dtype=np.int64)
    D = learn.shape[1]
    check_shape(D, T, M)
    h, s, m2 = D // 2, D // M, M // 2
    rot0 = rotations[0] if rotations is not None else opq_rotation(learn, 2)
    lp = round_half_up(learn @ rot0.T)
    C1, _ = kmeans(lp[:, :h], T, iters)
    C2, _ = kmeans(lp[:, h:], T, iters)
    i, j = coarse_cells(lp, C1, C2)
    disp = lp - np.concatenate([C1[i], C2[j]], axis=1)
    if rotations is not None:
        rot1, rot2 = rotations[1], rotations[2]
    else:
        rot1, rot2 = opq_rotation(disp[:, :h], m2), opq_rotation(disp[:, h:], m2)
    dr = np.concatenate([round_half_up(disp[:, :h] @ rot1.T), round_half_up(disp[:, h:] @ rot2.T)], axis=1)
    R = np.stack([kmeans(dr[:, k * s:(k + 1) * s], KSUB, iters)[0] for k in range(M)])
    return Codebooks(D=D, T=T, M=M, C1=C1, C2=C2, R=R, rot0=rot0, rot1=rot1, rot2=rot2)


def train_hbpq_local(learn, cb: Codebooks, iters):
    """HBPQ local codebooks of §3.2.  For each first-half Voronoi cell U_i (Eq. 10)
    the M/2 codebooks Q^i_k are learned on the displacements p^1 - c^1_i of the learn
    points falling in U_i (Eq. 11); S^j_k likewise on the second halves in V_j.
    Reading: each local codebook starts from the global R_k of the same
    sub-quantizer; a half-cell with no learn points keeps the global codebook."""
    learn = np.asarray(learn, dtype=np.int64)
    if cb.rotated:
        raise ValueError("local codebooks are built for unrotated codebooks")
    D, T, M, s = cb.D, cb.T, cb.M, cb.sub
    h, m2 = D // 2, M // 2
    i, j = coarse_cells(learn, cb.C1, cb.C2)
    Q = np.empty((T, m2, KSUB, s), dtype=np.int64)
    S = np.empty((T, m2, KSUB, s), dtype=np.int64)
    d1 = learn[:, :h] - cb.C1[i]
    d2 = learn[:, h:] - cb.C2[j]
    for cell in range(T):
        sel1, sel2 = d1[i == cell], d2[j == cell]
        for k in range(m2):
            Q[cell, k] = (kmeans(sel1[:, k * s:(k + 1) * s], KSUB, iters, init=cb.R[k])[0]
                          if len(sel1) else cb.R[k])
            S[cell, k] = (kmeans(sel2[:, k * s:(k + 1) * s], KSUB, iters, init=cb.R[m2 + k])[0]
                          if len(sel2) else cb.R[m2 + k])
    return dataclasses.replace(cb, Q=Q, S=S)


# ----------------------------------------------------------------------------
# Encoding and the inverted multi-index (§2.3.2, §3.2)
# ----------------------------------------------------------------------------


def encode_multi_d_adc(X, cb: Codebooks):
    """Cell and PQ code of each point (§2.3.2): d = x - [c^1_i; c^2_j] (Eq. 6) is
    encoded with R_1..R_M, code k = argmin_t ||d_k - R_k[t]||^2.  With OPQ rotations
    the cell comes from x' = rot0 x and the code from the rotated displacement
    [rot1 d^1; rot2 d^2] (FP64; no rounding of points)."""
    X = np.asarray(X, dtype=np.int64)
    s = cb.sub
    Xc = cb.coarse_space(X)
    i, j = coarse_cells(Xc, cb.C1, cb.C2)
    disp = cb.residual_space(Xc - np.concatenate([cb.C1[i], cb.C2[j]], axis=1))
    codes = np.stack([nearest(disp[:, k * s:(k + 1) * s], cb.R[k]) for k in range(cb.M)], axis=1)
    return i * cb.T + j, codes.astype(np.uint8)


def encode_hbpq(X, cb: Codebooks):
    """HBPQ encoding (Eq. 12): d^1 = p^1 - c^1_i is encoded with the local codebooks
    Q^i_1..Q^i_{M/2} and d^2 = p^2 - c^2_j with S^j_1..S^j_{M/2}."""
    X = np.asarray(X, dtype=np.int64)
    s, h, m2 = cb.sub, cb.D // 2, cb.M // 2
    i, j = coarse_cells(X, cb.C1, cb.C2)
    d1 = X[:, :h] - cb.C1[i]
    d2 = X[:, h:] - cb.C2[j]
    codes = np.empty((len(X), cb.M), dtype=np.uint8)
    for cell in np.unique(i):
        sel = np.nonzero(i == cell)[0]
        for k in range(m2):
            codes[sel, k] = nearest(d1[sel, k * s:(k + 1) * s], cb.Q[cell, k])
    for cell in np.unique(j):
        sel = np.nonzero(j == cell)[0]
        for k in range(m2):
            codes[sel, m2 + k] = nearest(d2[sel, k * s:(k + 1) * s], cb.S[cell, k])
    return i * cb.T + j, codes


@dataclasses.dataclass
class Lists:
    """Inverted multi-index storage (§2.3.2): the points of every cell stored
    contiguously in one array, cells in id order, plus the start of every cell."""
    T: int
    offsets: np.ndarray  # (T*T + 1,) int64
    codes: np.ndarray    # (N, M) uint8, cell-contiguous
    ids: np.ndarray      # (N,) int64, ascending inside a cell

    def counts(self):
        return np.diff(self.offsets)


def build_lists(cells, codes, ids, T):
    """Stable bucket order by cell id; ids ascending inside a cell."""
    cells = np.asarray(cells, dtype=np.int64)
    ids = np.asarray(ids, dtype=np.int64)
    order = np.lexsort((ids, cells))
    counts = np.bincount(cells, minlength=T * T)
    offsets = np.zeros(T * T + 1, dtype=np.int64)
    np.cumsum(counts, out=offsets[1:])
    return Lists(T=T, offsets=offsets, codes=np.asarray(codes)[order], ids=ids[order])


# ----------------------------------------------------------------------------
# Query side: coarse distances and traversal (§2.3.3)
# ----------------------------------------------------------------------------


def coarse_distances(q, cb: Codebooks):
    """d1[i] = ||q^1 - c^1_i||^2 and d2[j] = ||q^2 - c^2_j||^2 for one query (with OPQ,
    of q' = rot0 q)."""
    q = cb.coarse_space(np.asarray(q, dtype=np.float64))
    h = cb.D // 2
    return sq_dists(q[None, :h], cb.C1)[0], sq_dists(q[None, h:], cb.C2)[0]


def traverse_full_sort(d1, d2, counts, L):
    """Plain definition of the visit order (§2.3.3): all T^2 cells sorted by
    (d1[i] + d2[j], i*T + j); the visited cells are the shortest prefix whose
    point counts sum to at least L (every cell if the index holds fewer).
    Returns (visited cell ids in order, keys, number of candidate points L')."""
    if L < 1:
        raise ValueError("L must be at least 1")
    T = len(d1)
    key = (np.asarray(d1, np.float64)[:, None] + np.asarray(d2, np.float64)[None, :]).ravel()
    cid = np.arange(T * T, dtype=np.int64)
    order = np.lexsort((cid, key))
    csum = np.cumsum(np.asarray(counts)[order])
    stop = int(np.searchsorted(csum, L, side="left"))
    n = min(stop + 1, T * T)
    return order[:n], key[order[:n]], int(csum[n - 1])


def traverse_multisequence(d1, d2, counts, L):
    """The multi-sequence algorithm cited in §2.3.3 (Babenko & Lempitsky, CVPR 2012).

    Both coarse distance lists are sorted (ties by index).  A priority queue holds
    frontier pairs (u, v) of positions in the two sorted lists, keyed by
    (s1[u] + s2[v], cell id).  Each step pops the smallest pair and emits its cell;
    then (u+1, v) enters the queue if v == 0 or (u+1, v-1) was already emitted, and
    (u, v+1) enters if u == 0 or (u-1, v+1) was already emitted.  The walk stops as
    soon as the emitted cells hold at least L points.
    Returns the same triple as traverse_full_sort."""
    if L < 1:
        raise ValueError("L must be at least 1")
    d1 = np.asarray(d1, np.float64)
    d2 = np.asarray(d2, np.float64)
    T = len(d1)
    p1 = sorted(range(T), key=lambda i: (d1[i], i))
    p2 = sorted(range(T), key=lambda j: (d2[j], j))
    s1 = [d1[i] for i in p1]
    s2 = [d2[j] for j in p2]
    counts = np.asarray(counts)
    emitted = set()
    heap = [(s1[0] + s2[0], p1[0] * T + p2[0], 0, 0)]
    cells, keys, total = [], [], 0
    while heap and total < L:
        key, cid, u, v = heapq.heappop(heap)
        emitted.add((u, v))
        cells.append(cid)
        keys.append(key)
        total += int(counts[cid])
        if u + 1 < T and (v == 0 or (u + 1, v - 1) in emitted):
            heapq.heappush(heap, (s1[u + 1] + s2[v], p1[u + 1] * T + p2[v], u + 1, v))
        if v + 1 < T and (u == 0 or (u - 1, v + 1) in emitted):
            heapq.heappush(heap, (s1[u] + s2[v + 1], p1[u] * T + p2[v + 1], u, v + 1))
    return np.asarray(cells, dtype=np.int64), np.asarray(keys), total


def candidates(cells_visited, lists: Lists):
    """Positions (into the list arrays) of every point of the visited cells, in visit order."""
    off = lists.offsets
    parts = [np.arange(off[c], off[c + 1]) for c in cells_visited]
    return np.concatenate(parts) if parts else np.zeros(0, dtype=np.int64)


# ----------------------------------------------------------------------------
# Scoring: Multi-D-ADC reconstruction (§2.3.3), FBPQ (§3.1), HBPQ (§3.2)
# ----------------------------------------------------------------------------


def reconstruct(cb: Codebooks, cell, codes):
    """Approximation of Eq. 7: x ~ [c^1_i; c^2_j] + [r_1; ...; r_M] with global R_k.
    With OPQ rotations, in the original space: x ~ rot0^T ([c^1_i; c^2_j] +
    [rot1^T r^1; rot2^T r^2])."""
    cell = np.asarray(cell, dtype=np.int64)
    codes = np.asarray(codes, dtype=np.int64)
    i, j = cell // cb.T, cell % cb.T
    r = np.concatenate([cb.R[k][codes[:, k]] for k in range(cb.M)], axis=1)
    if cb.rotated:
        h = cb.D // 2
        r = np.concatenate([r[:, :h] @ cb.rot1, r[:, h:] @ cb.rot2], axis=1).astype(np.float64)
        return (np.concatenate([cb.C1[i], cb.C2[j]], axis=1).astype(np.float64) + r) @ cb.rot0
    return np.concatenate([cb.C1[i], cb.C2[j]], axis=1).astype(np.float64) + r


def reconstruct_hbpq(cb: Codebooks, cell, codes):
    """HBPQ approximation (§3.2): the displacement halves come from the local
    codebooks Q^i_k and S^j_k of the cell's two half-cells."""
    cell = np.asarray(cell, dtype=np.int64)
    codes = np.asarray(codes, dtype=np.int64)
    i, j = cell // cb.T, cell % cb.T
    m2 = cb.M // 2
    r1 = np.concatenate([cb.Q[i, k, codes[:, k]] for k in range(m2)], axis=1)
    r2 = np.concatenate([cb.S[j, k, codes[:, m2 + k]] for k in range(m2)], axis=1)
    return np.concatenate([cb.C1[i] + r1, cb.C2[j] + r2], axis=1).astype(np.float64)


def hbpq_tables(q, cb: Codebooks, i, j):
    """Per-query lookup tables of HBPQ for the half-cells i (first half) and j
    (second half): the O(D) reconstruction distance of §3.2 regrouped so that a
    point costs M lookups.  With r^1 = [Q^i_1[c_1] .. Q^i_{M/2}[c_{M/2}]],
        ||q^1 - c^1_i - r^1||^2 = ||q^1 - c^1_i||^2
                                  + sum_k ( ||Q^i_k[c_k]||^2 - 2 <q_k - c^1_i|k, Q^i_k[c_k]> )
    (c^1_i|k: block k of c^1_i), and likewise for the second half with S^j and c^2_j.
    Returns A (M/2, 256) and B (M/2, 256), FP64:
        A[k][t] = ||Q^i_k[t]||^2 + 2 <c^1_i|k, Q^i_k[t]> - 2 <q_k, Q^i_k[t]>
        B[k][t] = ||S^j_k[t]||^2 + 2 <c^2_j|k, S^j_k[t]> - 2 <q_{M/2+k}, S^j_k[t]>
    so that ||q - xhat||^2 = d1[i] + d2[j] + sum_k A[k][c_k] + sum_k B[k][c_{M/2+k}]."""
    q = np.asarray(q, np.float64)
    s, m2, h = cb.sub, cb.M // 2, cb.D // 2
    A = np.empty((m2, KSUB))
    B = np.empty((m2, KSUB))
    for k in range(m2):
        Qk = cb.Q[i, k].astype(np.float64)
        Sk = cb.S[j, k].astype(np.float64)
        c1 = cb.C1[i, k * s:(k + 1) * s].astype(np.float64)
        c2 = cb.C2[j, k * s:(k + 1) * s].astype(np.float64)
        A[k] = (Qk * Qk).sum(1) + 2.0 * (Qk @ c1) - 2.0 * (Qk @ q[k * s:(k + 1) * s])
        B[k] = (Sk * Sk).sum(1) + 2.0 * (Sk @ c2) - 2.0 * (Sk @ q[h + k * s:h + (k + 1) * s])
    return A, B


def dist_hbpq_tables(q, cb: Codebooks, cell, codes):
    """HBPQ distance of every point through hbpq_tables: d1[i] + d2[j] plus M
    lookups, one table pair per distinct half-cell pair (i, j)."""
    cell = np.asarray(cell, dtype=np.int64)
    codes = np.asarray(codes, dtype=np.int64)
    m2 = cb.M // 2
    d1, d2 = coarse_distances(q, cb)
    i, j = cell // cb.T, cell % cb.T
    out = np.empty(len(cell))
    for ii, jj in sorted(set(zip(i.tolist(), j.tolist()))):
        sel = (i == ii) & (j == jj)
        A, B = hbpq_tables(q, cb, ii, jj)
        c = codes[sel]
        out[sel] = (d1[ii] + d2[jj] + sum(A[k][c[:, k]] for k in range(m2))
                    + sum(B[k][c[:, m2 + k]] for k in range(m2)))
    return out


def dist_reconstruct(q, xhat):
    """Multi-D-ADC distance (§2.3.3): ||q - xhat||^2 from the explicit reconstruction, O(D) per point."""
    diff = np.asarray(q, np.float64)[None, :] - xhat
    return (diff * diff).sum(1)


@dataclasses.dataclass
class FbpqTables:
    """Query-independent FBPQ tables (Eq. 9, §3.3): squared norms of all
    codewords and the dot products of coarse and residual codewords."""
    n1: np.ndarray   # (T,)  ||c^1_i||^2
    n2: np.ndarray   # (T,)  ||c^2_j||^2
    nR: np.ndarray   # (M, 256)  ||R_k[t]||^2
    X1: np.ndarray   # (T, M/2, 256)  <c^1_i restricted to block k, R_k[t]>, k < M/2
    X2: np.ndarray   # (T, M/2, 256)  <c^2_j restricted to block k - M/2, R_k[t]>, k >= M/2


def fbpq_tables(cb: Codebooks):
    """With OPQ rotations the dot products of Eq. 9 are taken in the residual space,
    with the rotated coarse centroids [rot1 c^1_i], [rot2 c^2_j] (the norms are
    unchanged by the rotations)."""
    s, m2 = cb.sub, cb.M // 2
    C1 = cb.C1.astype(np.float64)
    C2 = cb.C2.astype(np.float64)
    R = cb.R.astype(np.float64)
    C1r, C2r = (np.asarray(c, np.float64) for c in cb.residual_centroids())
    X1 = np.stack([C1r[:, k * s:(k + 1) * s] @ R[k].T for k in range(m2)], axis=1)
    X2 = np.stack([C2r[:, k * s:(k + 1) * s] @ R[m2 + k].T for k in range(m2)], axis=1)
    return FbpqTables(n1=(C1 * C1).sum(1), n2=(C2 * C2).sum(1), nR=(R * R).sum(2), X1=X1, X2=X2)


def dist_fbpq(q, cb: Codebooks, tab: FbpqTables, cell, codes):
    """FBPQ distance, Eq. 8 with the query-independent term expanded by Eq. 9:

        ||q||^2 - 2<q, [c^1_i; c^2_j]> - 2<q, [r_1..r_M]>
          + ||c^1_i||^2 + ||c^2_j||^2 + sum_k ||r_k||^2
          + 2 sum_{k<=M/2} <c^1_i, r_k> + 2 sum_{k>M/2} <c^2_j, r_k>

    The query tables <q^1, c^1_i>, <q^2, c^2_j> and <q_k, R_k[t]> are built once
    per query (§3.1) and every term is then a lookup, O(M) per point.  With OPQ
    rotations the coarse terms use q' = rot0 q and the residual terms the rotated
    query [rot1 q'^1; rot2 q'^2] (the rotations are orthogonal, so the sum is the
    distance to the reconstruction in the original space)."""
    q = cb.coarse_space(np.asarray(q, np.float64))
    qr_vec = cb.residual_space(q)
    cell = np.asarray(cell, dtype=np.int64)
    codes = np.asarray(codes, dtype=np.int64)
    s, h, m2 = cb.sub, cb.D // 2, cb.M // 2
    i, j = cell // cb.T, cell % cb.T
    qc1 = cb.C1.astype(np.float64) @ q[:h]
    qc2 = cb.C2.astype(np.float64) @ q[h:]
    qr = np.stack([cb.R[k].astype(np.float64) @ qr_vec[k * s:(k + 1) * s] for k in range(cb.M)])
    ks = np.arange(cb.M)
    dot_qr = qr[ks[None, :], codes].sum(1)
    norm_r = tab.nR[ks[None, :], codes].sum(1)
    cross1 = sum(tab.X1[i, k, codes[:, k]] for k in range(m2))
    cross2 = sum(tab.X2[j, k, codes[:, m2 + k]] for k in range(m2))
    return ((q @ q) - 2.0 * (qc1[i] + qc2[j]) - 2.0 * dot_qr
            + tab.n1[i] + tab.n2[j] + norm_r + 2.0 * cross1 + 2.0 * cross2)


# ----------------------------------------------------------------------------
# Reduced-precision table with exact re-scoring (a precision variant of §3.1;
# the paper's own scan uses full-precision tables).  The score is formed in
# IEEE FP32 in a fixed order so that a GPU computing it the same way agrees bit
# for bit; everything else stays FP64.
# ----------------------------------------------------------------------------


def pq_table(q, cb: Codebooks):
    """Per-query PQ table of §3.1: lut[k][t] = ||R_k[t]||^2 - 2<q_k, R_k[t]>, the
    query term of Eq. 8 plus the codeword norm of Eq. 9, shape (M, 256) (with OPQ,
    of the rotated query [rot1 q'^1; rot2 q'^2], q' = rot0 q)."""
    q = cb.residual_space(cb.coarse_space(np.asarray(q, np.float64)))
    s = cb.sub
    R = cb.R.astype(np.float64)
    return np.stack([(R[k] * R[k]).sum(1) - 2.0 * (R[k] @ q[k * s:(k + 1) * s]) for k in range(cb.M)])


def point_cross(cb: Codebooks, tab: FbpqTables, cell, codes):
    """The query-independent cross terms of Eq. 9 for each point:
    2 sum_{k<=M/2} <c^1_i, r_k> + 2 sum_{k>M/2} <c^2_j, r_k>."""
    cell = np.asarray(cell, dtype=np.int64)
    codes = np.asarray(codes, dtype=np.int64)
    m2 = cb.M // 2
    i, j = cell // cb.T, cell % cb.T
    return 2.0 * (sum(tab.X1[i, k, codes[:, k]] for k in range(m2))
                  + sum(tab.X2[j, k, codes[:, m2 + k]] for k in range(m2)))


def quantize_table_int8(lut):
    """Per sub-quantizer offset lo_k = min_t lut[k][t] and one per-query step
    s = max_k (max_t lut[k][t] - lo_k) / 255 (1 when every table is constant);
    q8[k][t] = round_half_even((lut[k][t] - lo_k) / s) in [0, 255].  The table
    entries are integers below 2^24 (integer grid), so their FP32 copies are exact
    and only the division rounds.  Returns (q8 int64 (M, 256), s float32)."""
    lut32 = np.asarray(lut, np.float64).astype(np.float32)
    x = lut32 - lut32.min(axis=1)[:, None]
    rng = x.max()
    step = np.float32(rng) / np.float32(255.0) if rng > 0 else np.float32(1.0)
    q8 = np.clip(np.rint(x / step), 0, 255).astype(np.int64)
    return q8, np.float32(step)


FP16_MAX = 65504.0


def quantize_table_fp16(lut):
    """Per sub-quantizer offset lo_k = min_t lut[k][t] and one per-query step s, the
    smallest power of two >= 1 with max_k (max_t lut[k][t] - lo_k) <= 65504 s (the
    largest finite FP16 value), so the scaling is exact; h[k][t] = the FP16 value
    nearest to (lut[k][t] - lo_k) / s (ties to even).  Returns (h float16 (M, 256),
    s float32)."""
    lut32 = np.asarray(lut, np.float64).astype(np.float32)
    x = lut32 - lut32.min(axis=1)[:, None]
    rng = float(x.max())
    step = 1.0
    while rng > FP16_MAX * step:
        step *= 2.0
    h = (x / np.float32(step)).astype(np.float16)
    return h, np.float32(step)


def shortlist_part(q, cb, codes, precision):
    """The reduced-precision part of a shortlist score, in FP32: s * sum_k q8[k][c_k]
    (int8: an exact integer sum) or s * (((h[0][c_0] + h[1][c_1]) + ...) + h[M-1][c_{M-1}])
    (fp16: FP32 additions in sub-quantizer order)."""
    lut = pq_table(q, cb)
    cols = np.arange(cb.M)
    if precision == "int8":
        q8, step = quantize_table_int8(lut)
        return step * q8[cols[None, :], codes].sum(1).astype(np.float32)
    if precision == "fp16":
        h, step = quantize_table_fp16(lut)
        acc = np.zeros(len(codes), np.float32)
        for kk in range(cb.M):
            acc = acc + h[kk, codes[:, kk]].astype(np.float32)
        return step * acc
    raise ValueError(precision)


def search_shortlist_one(index: OracleIndex, q, L, k, S, precision="int8"):
    """One query of the reduced-precision table search: the visited cells and
    candidates of search_one; score = (key(i,j) + cross(p)) + part in FP32, part
    from shortlist_part (the constant sum_k lo_k is left out); the S best by
    (score, list position) are re-scored with the exact FBPQ distance (Eqs. 8-9)
    and ranked by (distance, id).  Returns (ids (k,), dists (k,))."""
    cb, lists, tab = index.cb, index.lists, index.tables
    if index.variant != "global":
        raise ValueError("the reduced-precision shortlist scores global codes")
    d1, d2 = coarse_distances(q, cb)
    cells, _, _ = traverse_full_sort(d1, d2, lists.counts(), L)
    pos = candidates(cells, lists)
    cell_of = np.repeat(cells, lists.counts()[cells])
    codes = lists.codes[pos].astype(np.int64)
    i, j = cell_of // cb.T, cell_of % cb.T
    key32 = (d1[i] + d2[j]).astype(np.float32)
    cross32 = point_cross(cb, tab, cell_of, codes).astype(np.float32)
    score = (key32 + cross32) + shortlist_part(q, cb, codes, precision)
    short = np.lexsort((pos, score))[:S]
    exact = dist_fbpq(q, cb, tab, cell_of[short], codes[short])
    return topk(exact, lists.ids[pos[short]], k)


def search_shortlist(index: OracleIndex, queries, L, k, S, precision="int8"):
    queries = np.asarray(queries)
    nq = len(queries)
    Ls = np.broadcast_to(np.asarray(L, dtype=np.int64), (nq,))
    ids = np.empty((nq, k), dtype=np.int64)
    dists = np.empty((nq, k))
    for n in range(nq):
        ids[n], dists[n] = search_shortlist_one(index, queries[n], int(Ls[n]), k, S, precision)
    return ids, dists


# ----------------------------------------------------------------------------
# Ranking, search, ground truth and recall
# ----------------------------------------------------------------------------


def topk(dists, ids, k):
    """The k smallest (distance, id) pairs in ascending order; pad with (+inf, -1)."""
    dists = np.asarray(dists, np.float64)
    ids = np.asarray(ids, np.int64)
    order = np.lexsort((ids, dists))[:k]
    out_d = np.full(k, np.inf)
    out_i = np.full(k, -1, dtype=np.int64)
    out_d[:len(order)] = dists[order]
    out_i[:len(order)] = ids[order]
    return out_i, out_d


SCORERS = ("fbpq", "recon", "hbpq", "hbpq_tables")


@dataclasses.dataclass
class OracleIndex:
    cb: Codebooks
    lists: Lists
    variant: str  # "global" (Multi-D-ADC / FBPQ codes) or "local" (HBPQ codes)
    tables: FbpqTables | None = None


def build_index(cb: Codebooks, X, ids=None, variant="global"):
    X = np.asarray(X)
    if ids is None:
        ids = np.arange(len(X), dtype=np.int64)
    if variant == "global":
        cells, codes = encode_multi_d_adc(X, cb)
        tab = fbpq_tables(cb)
    elif variant == "local":
        cells, codes = encode_hbpq(X, cb)
        tab = None
    else:
        raise ValueError(variant)
    return OracleIndex(cb=cb, lists=build_lists(cells, codes, ids, cb.T), variant=variant, tables=tab)


def search_one(index: OracleIndex, q, L, k, scorer="fbpq", traversal="multisequence", cut_counts=None):
    """One query of §2.3.3 / §3.1 / §3.2: coarse distances, traversal until L points,
    distances of all candidates with the chosen scorer, rerank by (distance, id).
    cut_counts: per-cell counts the stopping rule uses instead of the index's own
    (a shard of a larger index traverses with the whole index's counts).
    Returns (ids (k,), dists (k,), visited cell ids, L')."""
    cb, lists = index.cb, index.lists
    d1, d2 = coarse_distances(q, cb)
    walk = traverse_multisequence if traversal == "multisequence" else traverse_full_sort
    counts = lists.counts() if cut_counts is None else np.asarray(cut_counts)
    cells, _, total = walk(d1, d2, counts, L)
    pos = candidates(cells, lists)
    cell_of = np.repeat(cells, lists.counts()[cells])
    codes = lists.codes[pos]
    if scorer == "recon":
        if index.variant != "global":
            raise ValueError("recon scores global codes")
        dist = dist_reconstruct(q, reconstruct(cb, cell_of, codes))
    elif scorer == "fbpq":
        if index.variant != "global":
            raise ValueError("fbpq scores global codes")
        dist = dist_fbpq(q, cb, index.tables, cell_of, codes)
    elif scorer == "hbpq":
        if index.variant != "local":
            raise ValueError("hbpq scores local codes")
        dist = dist_reconstruct(q, reconstruct_hbpq(cb, cell_of, codes))
    elif scorer == "hbpq_tables":
        if index.variant != "local":
            raise ValueError("hbpq scores local codes")
        dist = dist_hbpq_tables(q, cb, cell_of, codes)
    else:
        raise ValueError(scorer)
    ids, dd = topk(dist, lists.ids[pos], k)
    return ids, dd, cells, total


def search(index: OracleIndex, queries, L, k, scorer="fbpq", traversal="multisequence"):
    queries = np.asarray(queries)
    nq = len(queries)
    Ls = np.broadcast_to(np.asarray(L, dtype=np.int64), (nq,))
    ids = np.empty((nq, k), dtype=np.int64)
    dists = np.empty((nq, k))
    totals = np.empty(nq, dtype=np.int64)
    for n in range(nq):
        ids[n], dists[n], _, totals[n] = search_one(index, queries[n], int(Ls[n]), k, scorer, traversal)
    return ids, dists, totals


def exact_nn(base, queries, chunk=4096):
    """True nearest neighbour of each query by brute force in exact int64
    arithmetic, ties to the lowest id (the ground truth behind Recall@T, §4)."""
    base = np.asarray(base, dtype=np.int64)
    out = np.empty(len(queries), dtype=np.int64)
    best = np.full(len(queries), np.iinfo(np.int64).max)
    for n, q in enumerate(np.asarray(queries, dtype=np.int64)):
        bd, bi = np.iinfo(np.int64).max, -1
        for s in range(0, len(base), chunk * 16):
            diff = base[s:s + chunk * 16] - q[None, :]
            d = (diff * diff).sum(1)
            m = int(np.argmin(d))
            if d[m] < bd:
                bd, bi = int(d[m]), s + m
        out[n], best[n] = bi, bd
    return out


def recall_at(result_ids, nn_ids, R):
    """Recall@R (§4): fraction of queries whose true nearest neighbour is among
    the first R returned ids."""
    result_ids = np.asarray(result_ids)
    return float(np.mean([nn_ids[n] in result_ids[n, :R] for n in range(len(nn_ids))]))


# ----------------------------------------------------------------------------
# Encoding error (§4.2, Fig. errors)
# ----------------------------------------------------------------------------


def encoding_error(cb: Codebooks, X, variant="global"):
    """Squared encoding error ||x - xhat||^2 of every point (§4.2, Fig. errors: the
    average of this over a dataset, with global codebooks (Eq. 7) or with the HBPQ
    local codebooks (§3.2)).  The point is encoded as the index encodes it
    (encode_multi_d_adc / encode_hbpq) and reconstructed from that code.
    Returns FP64 (n,); exact integers on the integer grid."""
    X = np.asarray(X, dtype=np.int64)
    if variant == "global":
        cells, codes = encode_multi_d_adc(X, cb)
        xhat = reconstruct(cb, cells, codes)
    elif variant == "local":
        cells, codes = encode_hbpq(X, cb)
        xhat = reconstruct_hbpq(cb, cells, codes)
    else:
        raise ValueError(variant)
    diff = X.astype(np.float64) - xhat
    return (diff * diff).sum(1)


# ----------------------------------------------------------------------------
# Memory accounting (§3.3)
# ----------------------------------------------------------------------------


def fbpq_table_floats(T, M, K=KSUB):
    """FBPQ dot-product tables: T*M*K floats (§3.3)."""
    return T * M * K


def fbpq_norm_floats(T, M, K=KSUB):
    """Codeword norms: 2T + M*K floats (§3.3)."""
    return 2 * T + M * K


def hbpq_local_floats(T, D, K=KSUB):
    """HBPQ local codebooks: T first-half cells x M/2 codebooks x K codewords x D/M
    dims, plus the same for the second half: T*K*D floats (§3.3, §4.2)."""
    return T * K * D
