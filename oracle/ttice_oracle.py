"""Plain FP64 CPU oracle for TT-ICE (Algorithm 1) and TT-ICE* (Algorithm 2) of arXiv 2211.12487.

TEST INFRASTRUCTURE ONLY.  This module is the reference the CUDA path is checked against.  Only the
test-suite, ``__graft_entry__.smoke()`` and the CPU-baseline leg of ``bench.py`` may import it; the
library itself never calls it and shares no code with it.

It is deliberately slow and literal: numpy in float64, one step of the paper per block of code, with
numpy's LAPACK SVD as the truncated-SVD primitive.  Nothing is fused, blocked or reordered beyond
what the algorithms state.

Conventions (the paper fixes none of them; each is a reading listed with the design notes):

* An increment is an array ``Y`` of shape ``(b, n_1, ..., n_d)``: ``b`` observations ("n_{d+1}^{k+1}"
  in the paper), each a d-way tensor, stored observation-major.
* Unfoldings use C order with the rank index slower than the mode index: row ``a*n_i + k`` of
  ``U_i`` is core entry ``G_i[a, k, :]`` (Eq. 3 reshape ``[r_{i-1}, n_i, r_i]``).  Padding a core
  (Eq. 11) therefore appends zero rows at the bottom.
* The stage-``i`` unfolding of a batch is held as ``(b, m_i, L_i)`` with ``m_i = r_{i-1} n_i`` and
  ``L_i = n_{i+1} ... n_d``; its matrix is the column concatenation of the b blocks.  Column order
  does not change a left singular subspace, a Gram matrix ``R R^T`` or a projection.
* The last core (Eq. 13) is a list of per-observation coefficient vectors; a vector appended when
  ``r_d`` was smaller is implicitly zero-extended (the padding of ``U_{d+1}``).
* New singular vectors are ordered by descending singular value, re-orthogonalised against the
  existing core by classical Gram-Schmidt applied twice (CGS2), and given a canonical sign: the entry
  of largest magnitude (lowest index on ties) is positive.
* Truncation (Eq. 5 tail bound, Eq. 9): the smallest ``r`` with ``sqrt(sum_{j>r} sigma_j^2) <= eps``.
* Per-core threshold (Corollary 1; Algorithm 2): ``eps_c = eps_upd * ||D||_F / sqrt(d)``.
* Skip modes (Sec. 4.3, last heuristic): ``exact`` skips iff the batch relative error (Eq. 20) is
  ``<= eps``; ``mean`` uses the paper's surrogate ``mean(eps_Y) <= eps``; ``none`` never skips.
* Subselection (Eqs. 17-18): ``D = {j : eps_Y(j) > eps}``; ``eps_upd`` exact (Eq. 18) or the
  count-weighted approximation (Eq. 19).  A zero-norm observation has ``eps_Y = 0``.
* Occupancy (Eq. 16): core ``i`` is left alone iff ``r_i / (r_{i-1} n_i) >= tau``.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

SKIP_NONE, SKIP_EXACT, SKIP_MEAN = 0, 1, 2
EPS_UPD_EXACT, EPS_UPD_APPROX = 0, 1


def truncation_rank(sigma: np.ndarray, tol: float) -> int:
    """Smallest r with sqrt(sum_{j>r} sigma_j^2) <= tol (Eckart-Young tail, Sec. 2.1 Eq. 5).

    ``sigma`` is sorted in descending order.  The tail sums are accumulated from the smallest
    singular value upward.
    """
    s2 = np.asarray(sigma, dtype=np.float64) ** 2
    n = s2.shape[0]
    tail = np.zeros(n + 1)
    for j in range(n - 1, -1, -1):
        tail[j] = tail[j + 1] + s2[j]
    for r in range(n + 1):
        if math.sqrt(tail[r]) <= tol:
            return r
    return n


def canonical_sign(V: np.ndarray) -> np.ndarray:
    """Flip each column so that its entry of largest magnitude (first on ties) is positive."""
    V = V.copy()
    for c in range(V.shape[1]):
        idx = int(np.argmax(np.abs(V[:, c])))
        if V[idx, c] < 0:
            V[:, c] = -V[:, c]
    return V


def cgs2_append(U: np.ndarray, V: np.ndarray) -> np.ndarray:
    """Orthonormalise the columns of V, one at a time, against [U, accepted columns] (CGS twice).

    Returns the new columns only (same count as V).  Used for the core expansion of Eq. 10, where
    the new left singular vectors must be orthogonal to the (padded) existing core.
    """
    Q = U.copy()
    out = []
    for c in range(V.shape[1]):
        v = V[:, c].copy()
        for _ in range(2):
            v = v - Q @ (Q.T @ v)
        v = v / np.linalg.norm(v)
        out.append(v)
        Q = np.concatenate([Q, v[:, None]], axis=1)
    return np.stack(out, axis=1) if out else np.zeros((U.shape[0], 0))


@dataclass
class UpdateStats:
    skipped: bool
    n_selected: int
    selected: list
    rel_err_before: float            # batch relative error against the old cores (Eq. 20)
    eps_upd: float
    eps_core: float
    ranks: list
    new_directions: list = field(default_factory=list)
    rel_err_after: float | None = None


class TTICEOracle:
    """State of an incremental TT decomposition: cores U_1..U_d and the growing last core."""

    def __init__(self, dims, eps: float, *, skip_mode: int = SKIP_EXACT, subselect: bool = True,
                 eps_upd_mode: int = EPS_UPD_EXACT, tau: float = 1.0):
        self.dims = [int(n) for n in dims]
        self.d = len(self.dims)
        self.eps = float(eps)
        self.skip_mode = int(skip_mode)
        self.subselect = bool(subselect)
        self.eps_upd_mode = int(eps_upd_mode)
        self.tau = float(tau)
        # ranks[i] = r_i for i = 0..d; r_0 = 1; all cores start empty (rank 0)
        self.ranks = [1] + [0] * self.d
        self.U = [np.zeros((self.dims[0], 0))] + [np.zeros((0, 0)) for _ in range(self.d - 1)]
        self.last: list[np.ndarray] = []

    # ------------------------------------------------------------------ helpers
    def m(self, i: int) -> int:
        """Rows of core i (0-based): r_{i-1} * n_i."""
        return self.ranks[i] * self.dims[i]

    def L(self, i: int) -> int:
        return int(np.prod(self.dims[i + 1:], dtype=np.int64)) if i + 1 < self.d else 1

    def _stage(self, X: np.ndarray, i: int) -> np.ndarray:
        """Reshape a (b, r_{i-1}, n_i * L_i) or (b, ...) array to the stage-i view (b, m_i, L_i)."""
        return X.reshape(X.shape[0], self.ranks[i] * self.dims[i], self.L(i))

    def project(self, Y: np.ndarray) -> np.ndarray:
        """Sequential projection onto U_1..U_d (Eq. 12, Algorithm 2 'project'): (b, r_d) coefficients."""
        Y = np.asarray(Y, dtype=np.float64)
        X = Y.reshape(Y.shape[0], self.dims[0], self.L(0))
        for i in range(self.d):
            W = np.einsum("mr,bml->brl", self.U[i], X)  # U_i^T Y_i for every observation
            if i + 1 < self.d:
                X = W.reshape(W.shape[0], self.ranks[i + 1] * self.dims[i + 1], self.L(i + 1))
            else:
                X = W
        return X.reshape(Y.shape[0], self.ranks[self.d])

    def expand(self, coeffs: np.ndarray) -> np.ndarray:
        """Contract cores U_1..U_d with coefficient vectors (Eq. 14): (b, r_d) -> (b, n_1, ..., n_d)."""
        C = np.asarray(coeffs, dtype=np.float64)
        b = C.shape[0]
        X = C.reshape(b, self.ranks[self.d], 1)
        for i in range(self.d - 1, -1, -1):
            # X: (b, r_{i+1}, rest) -> (b, r_i * n_i, rest) -> (b, r_i, n_i * rest)
            X = np.einsum("mr,brl->bml", self.U[i], X)
            X = X.reshape(b, self.ranks[i], self.dims[i] * self.L(i))
        return X.reshape((b,) + tuple(self.dims))

    def reconstruct(self, first: int, count: int) -> np.ndarray:
        """Reconstruct stored observations first..first+count-1 from the last core (Eq. 14)."""
        rd = self.ranks[self.d]
        C = np.zeros((count, rd))
        for j in range(count):
            c = self.last[first + j]
            C[j, :c.shape[0]] = c
        return self.expand(C)

    def last_core(self) -> np.ndarray:
        """The last core U_{d+1} as an r_d x (observations) matrix (Eq. 13, zero-padded columns)."""
        rd = self.ranks[self.d]
        M = np.zeros((rd, len(self.last)))
        for j, c in enumerate(self.last):
            M[:c.shape[0], j] = c
        return M

    def errors(self, Y: np.ndarray):
        """Per-observation squared errors rho_j^2 = ||y_j - ~y_j||^2 and norms ||y_j||^2 (Eq. 17)."""
        Y = np.asarray(Y, dtype=np.float64)
        b = Y.shape[0]
        coeffs = self.project(Y)
        approx = self.expand(coeffs)
        diff = (Y - approx).reshape(b, -1)
        rho2 = np.einsum("bi,bi->b", diff, diff)
        y2 = np.einsum("bi,bi->b", Y.reshape(b, -1), Y.reshape(b, -1))
        return coeffs, rho2, y2

    # ------------------------------------------------------------------ the update
    def update(self, Y: np.ndarray, check_error: bool = False) -> UpdateStats:
        """One TT-ICE* increment (Algorithm 2); with skip_mode=none, subselect off and tau=inf it is
        exactly TT-ICE (Algorithm 1)."""
        Y = np.asarray(Y, dtype=np.float64)
        assert Y.shape[1:] == tuple(self.dims), (Y.shape, self.dims)
        b = Y.shape[0]
        eps, d = self.eps, self.d

        # Per-observation relative errors against the current cores (Eq. 17).
        coeffs, rho2, y2 = self.errors(Y)
        rel = np.where(y2 > 0, np.sqrt(rho2 / np.where(y2 > 0, y2, 1.0)), 0.0)
        ynorm2 = float(y2.sum())
        batch_err = math.sqrt(float(rho2.sum()) / ynorm2) if ynorm2 > 0 else 0.0

        # Skip test (Eq. 20 exactly, or the paper's mean surrogate).
        if self.skip_mode == SKIP_EXACT:
            skip = batch_err <= eps
        elif self.skip_mode == SKIP_MEAN:
            skip = float(rel.mean()) <= eps
        else:
            skip = False

        stats = UpdateStats(skipped=bool(skip), n_selected=0, selected=[], rel_err_before=batch_err,
                            eps_upd=float("nan"), eps_core=float("nan"), ranks=[])
        if not skip:
            # Subselection (Eqs. 17-19).
            if self.subselect:
                sel = [j for j in range(b) if rel[j] > eps]
                rest = [j for j in range(b) if not rel[j] > eps]
            else:
                sel, rest = list(range(b)), []
            stats.selected = sel
            stats.n_selected = len(sel)
            if sel:
                dnorm2 = float(y2[sel].sum())
                if not rest:
                    eps_upd = eps
                elif self.eps_upd_mode == EPS_UPD_EXACT:
                    num = (eps * math.sqrt(ynorm2)) ** 2 - float(rho2[rest].sum())
                    eps_upd = math.sqrt(max(num, 0.0) / dnorm2)
                else:
                    eps_upd = (eps * b - float(rel[rest].sum())) / len(sel)
                    eps_upd = max(eps_upd, 0.0)
                eps_c = eps_upd * math.sqrt(dnorm2) / math.sqrt(d)
                stats.eps_upd, stats.eps_core = eps_upd, eps_c
                self._update_cores(Y[sel], eps_c, stats)
            coeffs = self.project(Y)

        # Append the coefficients of every observation to the last core (Eq. 13 / Eq. 21).
        for j in range(b):
            self.last.append(coeffs[j].copy())
        stats.ranks = list(self.ranks) + [1]
        if check_error:
            approx = self.expand(coeffs)
            stats.rel_err_after = (math.sqrt(float(((Y - approx) ** 2).sum()) / ynorm2)
                                   if ynorm2 > 0 else 0.0)
        return stats

    def _update_cores(self, D: np.ndarray, eps_c: float, stats: UpdateStats):
        """Core loop of Algorithm 2 (Algorithm 1 steps for each core i = 1..d) on the selected D."""
        d = self.d
        nD = D.shape[0]
        X = D.reshape(nD, self.dims[0], self.L(0))  # D_1
        for i in range(d):
            m_i = self.m(i)
            r_i = self.ranks[i + 1]
            U = self.U[i]
            grew = 0
            if not (r_i >= self.tau * m_i):  # occupancy r_i / (r_{i-1} n_i) below tau (Eq. 16)
                # Residual against the (padded) core (Eq. 6 / Eq. 12 with Alg. 1 indexing).
                W = np.einsum("mr,bml->brl", U, X)
                R = X - np.einsum("mr,brl->bml", U, W)
                Rmat = R.transpose(1, 0, 2).reshape(m_i, -1)
                # Truncated SVD of the residual (Eq. 9).
                Ur, s, _ = np.linalg.svd(Rmat, full_matrices=False)
                rR = min(truncation_rank(s, eps_c), m_i - r_i)
                if rR > 0:
                    new = canonical_sign(cgs2_append(U, Ur[:, :rR]))
                    self.U[i] = np.concatenate([U, new], axis=1)  # core expansion (Eq. 10)
                    self.ranks[i + 1] = r_i + rR
                    grew = rR
                    if i + 1 < d:  # zero-pad the next core (Eq. 11)
                        nxt = self.U[i + 1]
                        pad = np.zeros((rR * self.dims[i + 1], nxt.shape[1]))
                        self.U[i + 1] = np.concatenate([nxt, pad], axis=0)
            stats.new_directions.append(grew)
            # Project onto the updated core (Eq. 12): D_{i+1} = reshape(U_i^T D_i).
            W = np.einsum("mr,bml->brl", self.U[i], X)
            if i + 1 < d:
                X = W.reshape(nD, self.ranks[i + 1] * self.dims[i + 1], self.L(i + 1))

    # ------------------------------------------------------------------ metrics
    def core_elements(self) -> int:
        """Parameters of the compressed representation: sum_i r_{i-1} n_i r_i over the d+1 cores."""
        tot = sum(self.ranks[i] * self.dims[i] * self.ranks[i + 1] for i in range(self.d))
        return tot + self.ranks[self.d] * len(self.last)

    def compression_ratio(self) -> float:
        """CR of Eq. 22: elements of the accumulation over the parameters of its TT representation."""
        full = int(np.prod(self.dims, dtype=np.int64)) * len(self.last)
        return full / max(self.core_elements(), 1)


def tt_svd(X: np.ndarray, eps: float):
    """TT-SVD (Oseledets' Algorithm 1, recalled in Sec. 2.1) of a D-way array with per-unfolding
    threshold delta = eps ||X||_F / sqrt(D-1).  Returns (cores U_1..U_{D-1} as unfoldings, last
    core as an r_{D-1} x n_D matrix, ranks [r_0, .., r_D])."""
    X = np.asarray(X, dtype=np.float64)
    dims = X.shape
    D = len(dims)
    delta = eps * float(np.linalg.norm(X.ravel())) / math.sqrt(D - 1)
    ranks = [1]
    cores = []
    Z = X.reshape(dims[0], -1)
    for i in range(D - 1):
        U, s, Vt = np.linalg.svd(Z, full_matrices=False)
        r = max(truncation_rank(s, delta), 1)
        cores.append(U[:, :r])
        ranks.append(r)
        Z = (s[:r, None] * Vt[:r])
        if i + 1 < D - 1:
            Z = Z.reshape(r * dims[i + 1], -1)
    ranks.append(1)
    return cores, Z, ranks
