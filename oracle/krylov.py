"""Sylvester operator, tArnoldi, tFOM and tGMRES (§3).  Oracle: test infrastructure only.

Readings of the paper taken here (the CUDA library follows the same ones):
  * M(X) = A*X - X*B, the form of Eq. (2) (the "+" of the STE in §2 and of
    Theorem 2.1 is read as a sign slip).
  * The stopping test is relative: ||C - M(X)||_F <= tol * ||C||_F.  The
    residual estimate is checked after every inner step; an inner cycle ends
    early when it passes, and a cycle's result is accepted only when the true
    residual passes too (otherwise the method restarts).
  * "Go to Step 2" in Algorithm 3 restarts from R0 = C - M(X0) with X0 <- Xm.
  * Arnoldi breakdown ("h_{j+1,j} = 0") is h_{j+1,j} <= 1e-14 * beta.
  * The tGMRES least-squares problem is solved as stated (a least-squares
    solve of the (j+1) x j Hessenberg system); its residual norm is the
    estimate |gamma_{j+1}| of Proposition 3.4.
  * tFOM solves H_j y = beta e1 and estimates h_{j+1,j} |y_j| (Proposition 3.3).
"""
from __future__ import annotations

import dataclasses
from typing import Callable, Optional

import numpy as np

from .tproduct import tprod, inner, norm

BREAKDOWN_REL = 1e-14


def sylv_apply(A: np.ndarray, B: np.ndarray, X: np.ndarray) -> np.ndarray:
    """The Sylvester operator of Eq. (2): M(X) = A*X - X*B."""
    return tprod(A, X) - tprod(X, B)


def tarnoldi(apply: Callable, V: np.ndarray, m: int):
    """Algorithm 2 (tArnoldi) on the operator `apply`.

    Returns (Vs, Htilde, beta): the basis tensors V_1..V_{k+1}, the (k+1) x k
    Hessenberg matrix and beta = ||V||_F; k < m only on breakdown.
    """
    beta = norm(V)
    Vs = [V / beta]
    H = np.zeros((m + 1, m))
    for j in range(m):
        W = apply(Vs[j])
        for i in range(j + 1):
            H[i, j] = inner(Vs[i], W)
            W = W - H[i, j] * Vs[i]
        H[j + 1, j] = norm(W)
        if H[j + 1, j] <= BREAKDOWN_REL * beta:
            return Vs, H[:j + 2, :j + 1], beta
        Vs.append(W / H[j + 1, j])
    return Vs, H, beta


def gmres_small(Ht: np.ndarray, beta: float):
    """tGMRES small problem: y = argmin || beta e1 - Htilde y ||_2 and that minimum."""
    rhs = np.zeros(Ht.shape[0])
    rhs[0] = beta
    y = np.linalg.lstsq(Ht, rhs, rcond=None)[0]
    return y, float(np.linalg.norm(rhs - Ht @ y))


def fom_small(Ht: np.ndarray, beta: float):
    """tFOM small problem: H_k y = beta e1, estimate h_{k+1,k} |y_k| (Proposition 3.3)."""
    k = Ht.shape[1]
    rhs = np.zeros(k)
    rhs[0] = beta
    y = np.linalg.solve(Ht[:k, :k], rhs)
    return y, float(abs(Ht[k, k - 1]) * abs(y[k - 1]))


@dataclasses.dataclass
class SolveResult:
    X: np.ndarray
    history: list          # residual estimate after every inner step (absolute)
    true_res: list         # ||C - M(X)||_F: initial, then after every cycle (absolute)
    iters: int             # inner steps taken
    cycles: int            # restart cycles run
    status: str            # "ok" | "not_converged" | "breakdown"
    normC: float

    @property
    def relres(self) -> float:
        return self.true_res[-1] / self.normC


def restarted_solve(method: str, A, B, C, X0=None, m: int = 20, tol: float = 1e-10,
                    max_restarts: int = 200, apply: Optional[Callable] = None) -> SolveResult:
    """Algorithm 3: restarted tFOM ("fom") or tGMRES ("gmres") for M(X) = C."""
    if apply is None:
        apply = lambda X: sylv_apply(A, B, X)  # noqa: E731
    small = gmres_small if method == "gmres" else fom_small
    X = np.zeros_like(C, dtype=float) if X0 is None else np.array(X0, dtype=float)
    normC = norm(C)
    R = C - apply(X)                                   # step 3
    res = norm(R)
    history, true_res = [], [res]
    iters = 0
    if res <= tol * normC:
        return SolveResult(X, history, true_res, 0, 0, "ok", normC)
    for cycle in range(max_restarts):                  # step 4
        beta = res
        Vs = [R / beta]
        H = np.zeros((m + 1, m))
        k, broke, y = 0, False, None
        for j in range(m):                             # step 4a: Algorithm 2, one step at a time
            W = apply(Vs[j])
            for i in range(j + 1):
                H[i, j] = inner(Vs[i], W)
                W = W - H[i, j] * Vs[i]
            H[j + 1, j] = norm(W)
            k = j + 1
            broke = H[j + 1, j] <= BREAKDOWN_REL * beta
            y, est = small(H[:k + 1, :k], beta)        # step 4b on the first k columns
            history.append(est)
            if est <= tol * normC or broke:
                break
            Vs.append(W / H[j + 1, j])
        X = X + sum(y[i] * Vs[i] for i in range(k))    # step 4c: X0 + V_k (*) y
        iters += k
        R = C - apply(X)                               # step 5: true residual
        res = norm(R)
        true_res.append(res)
        if res <= tol * normC:
            return SolveResult(X, history, true_res, iters, cycle + 1, "ok", normC)
        if broke:
            return SolveResult(X, history, true_res, iters, cycle + 1, "breakdown", normC)
    return SolveResult(X, history, true_res, iters, max_restarts, "not_converged", normC)


def tgmres(A, B, C, X0=None, m=20, tol=1e-10, max_restarts=200, apply=None) -> SolveResult:
    """Restarted tGMRES(m) (§3.3, Algorithm 3)."""
    return restarted_solve("gmres", A, B, C, X0, m, tol, max_restarts, apply)


def tfom(A, B, C, X0=None, m=20, tol=1e-10, max_restarts=200, apply=None) -> SolveResult:
    """Restarted tFOM(m) (§3.2, Algorithm 3)."""
    return restarted_solve("fom", A, B, C, X0, m, tol, max_restarts, apply)


def combine(Vs, y) -> np.ndarray:
    """The (*) product of §3.1: V_m (*) y = sum_j y_j V_j."""
    return sum(y[j] * Vs[j] for j in range(len(y)))
