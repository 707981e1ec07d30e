"""FP64 oracle of the NMPBB iteration and its symmetric variants.

TEST INFRASTRUCTURE ONLY (see the package docstring).

Notation follows the paper: V is the symmetric input (called A here), W the left
factor, H the right factor (stored transposed as Ht = H^T, n x r), lambda the
symmetric penalty weight, gamma the graph weight, L the graph Laplacian.

Formulations
* "penalty" (SNMPBB, Sec. 2.1): f(W,H) = 1/2 ||V - W H||^2 + lambda/2 ||W - H^T||^2
  (Eq. (3)), plus gamma/2 tr(H L H^T) for Graph-SNMPBB (Eq. (5)), minimised by
  alternating Algorithm 1 over the W block and the H block with the gradients of
  Eqs. (2.1)-(2.2) (and the graph gradient of Sec. 2.2).
* "direct": the single-variable objective of Eq. (2) with the 1/4 scaling that
  makes W (W^T W) - V W its exact gradient, plus gamma/2 tr(W^T L W), minimised by
  Algorithm 1 with rho_k = 3 ||W_k^T W_k||_2 recomputed at every step (see
  ``snmpbb_direct`` for this reading).

The oracle evaluates f by its definition (forming V - W H^T) unless
``objective="closed"`` is requested, which uses the Frobenius expansion; the two
agreeing is itself one of the pins.
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np


@dataclasses.dataclass
class Options:
    """Method parameters (Algorithm 1 REQUIRE line; Sec. 2.4; Sec. 4.1)."""

    formulation: str = "penalty"  # "penalty" | "direct"
    lambda_sym: float = -1.0      # < 0: 0.01 ||V||_F (Sec. 4.1 guideline (1))
    gamma: float = 0.0            # graph weight (Eq. (5))
    theta: float = 1e-3           # Armijo parameter (Sec. 2.4)
    phi: float = 1.7              # relaxation factor (Sec. 2.4)
    eta: float = 0.85             # averaging weight of F_k (reading: paper gives none)
    memory: int = 0               # 0: eta averaging of Alg. 1; M > 0: max of last M values
    bb: str = "bb1"               # "bb1": <S,S>/<S,Y> (Alg. 1, Eq. (2.10)); "bb2": <S,Y>/<Y,Y>
    alpha_min: float = 1e-10      # reading: paper gives no values
    alpha_max: float = 1e10
    beta_shrink: float = 0.5      # backtracking factor (reading)
    max_ls: int = 20              # line-search trials (Sec. 4.1 guideline (5))
    inner_iters: int = 5          # K of each block (reading; 3-5 in Sec. 4.4)
    max_iter: int = 500           # outer iterations (penalty) or steps (direct)
    tol: float = 1e-4             # relative projected-gradient tolerance
    power_iters: int = 50         # iterations of the rho_0 power method
    direct_rho_factor: float = 3.0  # direct form: rho_k = factor * ||W_k^T W_k||_2 (reading)
    objective: str = "explicit"   # "explicit" | "closed"


@dataclasses.dataclass
class LaiOperator:
    """Low-rank approximate input V ~ U diag(lam) U^T (Sec. 2.3, Eq. (8))."""

    U: np.ndarray
    lam: np.ndarray


def apply_A(A, X: np.ndarray) -> np.ndarray:
    """V X; for the LAI operator U E (U^T X) with U^T X formed first (Sec. 2.3)."""
    if isinstance(A, LaiOperator):
        return A.U @ (A.lam[:, None] * (A.U.T @ X))
    return A @ X


def dense_of(A) -> np.ndarray:
    if isinstance(A, LaiOperator):
        return (A.U * A.lam[None, :]) @ A.U.T
    return np.asarray(A, dtype=np.float64)


def proj(X: np.ndarray) -> np.ndarray:
    """Proj[X]: elementwise max(X, 0) (Sec. 1.1, Notation)."""
    return np.where(X >= 0.0, X, 0.0)


def inner(X: np.ndarray, Y: np.ndarray) -> float:
    """Frobenius inner product <X, Y> = sum_ij X_ij Y_ij (Sec. 1.1)."""
    return float(np.sum(X * Y))


def spectral_norm(G: np.ndarray, iters: int = 50) -> float:
    """||G||_2 of a symmetric PSD Gram matrix, used for rho_0 (Alg. 1 line 2, Eq. (2.11)).

    Reading: a fixed number of power iterations from the all-ones vector followed
    by the Rayleigh quotient.  The Gram of a nonnegative factor is entrywise
    nonnegative, so its Perron vector has a positive overlap with the start.
    """
    r = G.shape[0]
    v = np.ones(r) / math.sqrt(r)
    for _ in range(iters):
        w = G @ v
        nw = float(np.linalg.norm(w))
        if nw == 0.0:
            return 0.0
        v = w / nw
    return float(v @ (G @ v))


def projected_gradient(X: np.ndarray, g: np.ndarray) -> np.ndarray:
    """Projected gradient: g_ij where X_ij > 0, else min(0, g_ij) (reading of the
    stopping test; the paper does not state one)."""
    return np.where(X > 0.0, g, np.minimum(g, 0.0))


def resolve_lambda(A, opts: Options) -> float:
    """lambda < 0 selects 0.01 ||V||_F (Sec. 4.1, guideline (1))."""
    if opts.lambda_sym >= 0.0:
        return float(opts.lambda_sym)
    return 0.01 * float(np.linalg.norm(dense_of(A)))


def svd_init(A, r: int):
    """SVD start of Sec. 4.1 guideline (4), recommended there for graph problems: with
    V ~ U E P^T (the r largest singular values), W_0 = |U E^(1/2)| and H_0 = |E^(1/2) P^T|.
    Returns (W0, Ht0), Ht0 = H_0^T = |P E^(1/2)|.  The absolute values make the start
    nonnegative and independent of the sign of each singular-vector pair.  For a symmetric
    V, P = U up to the signs of V's eigenvalues, so W0 = Ht0."""
    V = dense_of(A)
    U, s, Pt = np.linalg.svd(V)
    e = np.sqrt(s[:r])
    W0 = np.abs(U[:, :r] * e[None, :])
    Ht0 = np.abs(Pt[:r, :].T * e[None, :])
    return W0, Ht0


def paper_laplacian(A) -> np.ndarray:
    """L = I - D^-1/2 V D^-1/2 with d_ii = e_i^T V e (Sec. 2.2).

    Reading: rows with zero degree get a zero scaling."""
    V = dense_of(A)
    d = V.sum(axis=1)
    s = np.where(d > 0.0, 1.0 / np.sqrt(np.where(d > 0.0, d, 1.0)), 0.0)
    return np.eye(V.shape[0]) - (s[:, None] * V) * s[None, :]


# ----------------------------------------------------------------------------
# Objectives and gradients
# ----------------------------------------------------------------------------

def direct_objective(A, X, gamma=0.0, L=None, mode="explicit") -> float:
    """1/4 ||V - X X^T||^2 (+ gamma/2 tr(X^T L X)): Eq. (2) scaled so that its
    gradient is X (X^T X) - V X."""
    if mode == "explicit":
        R = dense_of(A) - X @ X.T
        f = 0.25 * float(np.sum(R * R))
    else:
        G = X.T @ X
        f = 0.25 * (frob2(A) - 2.0 * inner(X, apply_A(A, X)) + float(np.sum(G * G)))
    if gamma != 0.0 and L is not None:
        f += 0.5 * gamma * inner(X, L @ X)
    return f


def direct_gradient(A, X, gamma=0.0, L=None) -> np.ndarray:
    g = X @ (X.T @ X) - apply_A(A, X)
    if gamma != 0.0 and L is not None:
        g = g + gamma * (L @ X)
    return g


def frob2(A) -> float:
    """||V||_F^2; for the LAI operator sum(lam^2) since U is orthonormal."""
    if isinstance(A, LaiOperator):
        return float(np.sum(A.lam * A.lam))
    return float(np.sum(A * A))


def penalty_objective(A, W, Ht, lam, gamma=0.0, L=None, mode="explicit") -> float:
    """f(W, H; lambda, gamma) of Eq. (3) / Eq. (5) with H = Ht^T."""
    if mode == "explicit":
        R = dense_of(A) - W @ Ht.T
        f = 0.5 * float(np.sum(R * R))
    else:
        f = 0.5 * frob2(A) - inner(W, apply_A(A, Ht)) + 0.5 * float(np.sum((W.T @ W) * (Ht.T @ Ht)))
    E = W - Ht
    f += 0.5 * lam * float(np.sum(E * E))
    if gamma != 0.0 and L is not None:
        f += 0.5 * gamma * inner(Ht, L @ Ht)
    return f


def penalty_grad_W(A, W, Ht, lam) -> np.ndarray:
    """Eq. (2.1): W H H^T - V H^T + lambda W - lambda H^T, with Ht = H^T."""
    return W @ (Ht.T @ Ht) - apply_A(A, Ht) + lam * W - lam * Ht


def penalty_grad_Ht(A, W, Ht, lam, gamma=0.0, L=None) -> np.ndarray:
    """Transpose of Eq. (2.2) (and of the Graph-SNMPBB H gradient of Sec. 2.2):
    (W^T W H - W^T V + lambda H - lambda W^T + gamma H L)^T
    = Ht W^T W - V W + lambda Ht - lambda W + gamma L Ht  (V, L symmetric)."""
    g = Ht @ (W.T @ W) - apply_A(A, W) + lam * Ht - lam * W
    if gamma != 0.0 and L is not None:
        g = g + gamma * (L @ Ht)
    return g


# ----------------------------------------------------------------------------
# Algorithm 1 (NMPBB) for one block
# ----------------------------------------------------------------------------

def laplacian_norm(L, iters: int = 50) -> float:
    """||L||_2 of the (positive semidefinite) graph Laplacian: the part gamma ||L||_2 that the
    graph term adds to the Lipschitz constant of the regularised block's gradient.

    Reading (the paper gives rho_0 = ||H H^T||_2 only for the unregularised blocks,
    Sec. 2.4): the graph-regularised blocks use rho = ||X^T X||_2 + gamma ||L||_2; without
    the gamma ||L||_2 part the first Z step of the 20000-point kNN workload (||L||_2 = 27,
    gamma = 0.1) overshoots and the iteration diverges.  Fixed count of power iterations
    from s_i = 1 + (i mod 2) (not constant: L 1 = 0) and the Rayleigh quotient."""
    n = L.shape[0]
    v = 1.0 + (np.arange(n) % 2).astype(np.float64)
    v /= np.linalg.norm(v)
    for _ in range(iters):
        w = np.asarray(L @ v).ravel()
        nw = float(np.linalg.norm(w))
        if nw == 0.0:
            return 0.0
        v = w / nw
    return float(v @ np.asarray(L @ v).ravel())


def _bb_step(S, Y, rho: float, opts: Options) -> float:
    """Alg. 1 line 3 / Eq. (2.10): alpha = min(a_max, max(a_min, <S,S>/<S,Y>)).

    Readings: "bb2" uses <S,Y>/<Y,Y>.  When <S,Y> <= 0 (no curvature along S; it
    cannot happen in the convex penalty blocks, where Y = S (H H^T + lambda I) by
    Sec. 3.3, but it does where the single-variable quartic is nonconvex) the
    step falls back to the Lipschitz-based 1/rho of the same iteration."""
    ss, sy, yy = inner(S, S), inner(S, Y), inner(Y, Y)
    if sy <= 0.0:
        a = 1.0 / rho
    else:
        a = ss / sy if opts.bb == "bb1" else sy / yy
    return min(opts.alpha_max, max(opts.alpha_min, a))


def nmpbb(fobj, fgrad, X0, rho_fn, K: int, opts: Options, stop_fn=None,
          keep_iterates=False):
    """Algorithm 1 for one block.

    Steps per iteration k (Alg. 1 lines 2-4):
      Z_k = Proj[X_k - grad f(X_k) / rho]                       (line 2, Eq. (2.11))
      alpha_k = clamp(BB(S_{k-1}, Y_{k-1}))   (k = 0: 1/rho, reading)  (line 3)
        (S/Y history and F restart with every call, i.e. every block, reading)
      D_k = Proj[Z_k - alpha_k grad f(Z_k)] - Z_k                (line 3)
      F_0 = f(X_0); F_k = f(X_k) + eta (F_{k-1} - f(X_k))         (line 4)
        (memory M > 0: F_k = max of the last M values f(X_k), ..., reading)
      beta = 1, shrink by beta_shrink until
        f(Z_k + beta D_k) <= F_k + theta beta <grad f(Z_k), D_k>  (line 4, Sec. 2.4)
        (max_ls trials; none accepted -> beta = 0, reading)
      X_{k+1} = Proj[Z_k + phi beta D_k]   (line 4; the projection keeps the
        relaxed point feasible when phi beta > 1, reading)
    ``rho_fn(X_k)`` returns rho (fixed rho_0 for the penalty blocks, ||X_k^T X_k||_2
    for the direct form).  ``stop_fn(X, g)`` is checked after every step.
    Returns (X, g, info).
    """
    X = np.array(X0, dtype=np.float64, copy=True)
    g = fgrad(X)
    fX = fobj(X)
    F = fX
    fhist = [fX]
    S = Y = None
    trace = []
    ls_fail = 0
    for k in range(K):
        rho = rho_fn(X)
        rho_eff = rho if rho > 0.0 else 1.0  # reading: zero Gram -> unit scaling
        Z = proj(X - g / rho_eff)
        gZ = fgrad(Z)
        alpha = 1.0 / rho_eff if k == 0 else _bb_step(S, Y, rho_eff, opts)
        D = proj(Z - alpha * gZ) - Z
        gd = inner(gZ, D)
        if k > 0:
            if opts.memory > 0:
                F = max(fhist[-opts.memory:])
            else:
                F = fX + opts.eta * (F - fX)
        beta = 1.0
        nls = 0
        accepted = False
        for t in range(opts.max_ls):
            nls = t + 1
            if fobj(Z + beta * D) <= F + opts.theta * beta * gd:
                accepted = True
                break
            beta *= opts.beta_shrink
        if not accepted:
            beta = 0.0
            ls_fail += 1
        Xn = proj(Z + opts.phi * beta * D)
        gn = fgrad(Xn)
        fn = fobj(Xn)
        S = Xn - X
        Y = gn - g
        rec = dict(k=k, rho=rho, alpha=alpha, beta=beta, nls=nls, F=F, f=fX, f_next=fn,
                   gd=gd, dd=inner(D, D), clipped=int(np.count_nonzero(Z + opts.phi * beta * D < 0.0)))
        if keep_iterates:
            rec["X"] = Xn.copy()
            rec["Z"] = Z.copy()
            rec["D"] = D.copy()
        trace.append(rec)
        X, g, fX = Xn, gn, fn
        fhist.append(fn)
        if stop_fn is not None and stop_fn(X, g):
            break
    return X, g, dict(trace=trace, ls_fail=ls_fail, f=fX)


# ----------------------------------------------------------------------------
# Drivers
# ----------------------------------------------------------------------------

def snmpbb_direct(A, W0, opts: Options, L=None, keep_iterates=False):
    """Algorithm 1 applied to the single-variable objective (see module docstring).

    Reading of rho for this form: the paper's rho_0 = ||H H^T||_2 is the Lipschitz
    constant of the block gradient (Sec. 2.4, Sec. 3.1).  For 1/4 ||V - W W^T||^2 the
    Hessian at W acts as E -> E W^T W + W E^T W + W W^T E - V E, whose largest
    eigenvalue is at most 3 ||W^T W||_2 when V is positive semidefinite, so
    rho_k = 3 ||W_k^T W_k||_2 (``direct_rho_factor``).  With the unscaled
    ||W_k^T W_k||_2 the first trial step maps a factor c W* to W*/c and the
    relaxed update drives a small start to W = 0.

    Stops when ||P grad f(W_k)||_F <= tol ||P grad f(W_0)||_F or after max_iter
    steps.  Returns (W, info) with info["trace"] holding one record per step."""
    gamma = opts.gamma
    mode = opts.objective

    def fobj(X):
        return direct_objective(A, X, gamma, L, mode)

    def fgrad(X):
        return direct_gradient(A, X, gamma, L)

    lshift = gamma * laplacian_norm(L, opts.power_iters) if (gamma and L is not None) else 0.0

    def rho_fn(X):
        return opts.direct_rho_factor * spectral_norm(X.T @ X, opts.power_iters) + lshift

    W0 = np.asarray(W0, dtype=np.float64)
    pg0 = float(np.linalg.norm(projected_gradient(W0, fgrad(W0))))

    def stop_fn(X, g):
        return float(np.linalg.norm(projected_gradient(X, g))) <= opts.tol * pg0

    W, g, info = nmpbb(fobj, fgrad, W0, rho_fn, opts.max_iter, opts, stop_fn, keep_iterates)
    info["iters"] = len(info["trace"])
    info["pg0"] = pg0
    info["pg"] = float(np.linalg.norm(projected_gradient(W, g)))
    Ad = dense_of(A)
    info["residual"] = float(np.linalg.norm(Ad - W @ W.T) / np.linalg.norm(Ad))
    return W, info


def snmpbb_naive(A, W0, opts: Options, keep_iterates=False):
    """The naive symmetric use of NMPBB that the paper describes before the penalty form
    (Sec. 2.1): each outer iteration runs Algorithm 1 on the W block of 1/2 ||V - W H||^2 with
    H = W^T held fixed (the NMF objective: no penalty term, rho_0 = ||W^T W||_2), then sets
    H <- W^T, i.e. Ht = W.

    Stopping reading (the paper gives none for this variant): the projected gradient of the
    W block at (W, H = W^T) relative to its value at W_0, after every outer iteration.
    Returns (W, info) with one iterate record per outer iteration."""
    zero = dataclasses.replace(opts, lambda_sym=0.0, gamma=0.0)
    mode = opts.objective
    W = np.array(W0, dtype=np.float64, copy=True)

    def pg_of(W):
        return float(np.linalg.norm(projected_gradient(W, penalty_grad_W(A, W, W, 0.0))))

    pg0 = pg_of(W)
    outer = []
    ls_fail = 0
    pg = pg0
    for it in range(1, opts.max_iter + 1):
        Hfix = W
        rho = spectral_norm(Hfix.T @ Hfix, opts.power_iters)
        W, _, iw = nmpbb(lambda X: penalty_objective(A, X, Hfix, 0.0, 0.0, None, mode),
                         lambda X: penalty_grad_W(A, X, Hfix, 0.0),
                         W, lambda X: rho, opts.inner_iters, zero, None, keep_iterates)
        ls_fail += iw["ls_fail"]
        pg = pg_of(W)
        rec = dict(i=it, rho=rho, pg=pg, w_trace=iw["trace"], f=penalty_objective(A, W, W, 0.0, 0.0, None, mode))
        if keep_iterates:
            rec["W"] = W.copy()
        outer.append(rec)
        if pg <= opts.tol * pg0:
            break
    Ad = dense_of(A)
    info = dict(trace=outer, iters=len(outer), pg0=pg0, pg=pg, ls_fail=ls_fail,
                residual=float(np.linalg.norm(Ad - W @ W.T) / np.linalg.norm(Ad)))
    return W, info


def snmpbb_penalty(A, W0, Ht0, opts: Options, L=None, keep_iterates=False):
    """SNMPBB / Graph-SNMPBB (Sec. 2.1-2.2): alternate Algorithm 1 over the W block
    (rho_0 = ||H H^T||_2 = ||Ht^T Ht||_2, lambda omitted, Eq. (2.11)) and the H block
    (rho_0 = ||W^T W||_2), ``inner_iters`` steps each.

    Stopping reading: the joint projected gradient (W and Ht blocks at the same
    point) relative to its value at (W_0, Ht_0), checked after every outer
    iteration.  Returns (W, Ht, info) with one iterate record per outer iteration.
    """
    lam = resolve_lambda(A, opts)
    gamma = opts.gamma
    mode = opts.objective
    W = np.array(W0, dtype=np.float64, copy=True)
    Ht = np.array(Ht0, dtype=np.float64, copy=True)

    def joint_pg(W, Ht):
        gW = penalty_grad_W(A, W, Ht, lam)
        gH = penalty_grad_Ht(A, W, Ht, lam, gamma, L)
        a = projected_gradient(W, gW)
        b = projected_gradient(Ht, gH)
        return math.sqrt(float(np.sum(a * a)) + float(np.sum(b * b)))

    pg0 = joint_pg(W, Ht)
    # graph term: gamma ||L||_2 joins rho of the H block (reading, see laplacian_norm)
    lshift = gamma * laplacian_norm(L, opts.power_iters) if (gamma and L is not None) else 0.0
    outer = []
    ls_fail = 0
    pg = pg0
    it = 0
    for it in range(1, opts.max_iter + 1):
        Hfix = Ht
        rho_w = spectral_norm(Hfix.T @ Hfix, opts.power_iters)
        W, _, iw = nmpbb(lambda X: penalty_objective(A, X, Hfix, lam, gamma, L, mode),
                         lambda X: penalty_grad_W(A, X, Hfix, lam),
                         W, lambda X: rho_w, opts.inner_iters, opts, None, keep_iterates)
        Wfix = W
        rho_h = spectral_norm(Wfix.T @ Wfix, opts.power_iters) + lshift
        Ht, _, ih = nmpbb(lambda X: penalty_objective(A, Wfix, X, lam, gamma, L, mode),
                          lambda X: penalty_grad_Ht(A, Wfix, X, lam, gamma, L),
                          Ht, lambda X: rho_h, opts.inner_iters, opts, None, keep_iterates)
        ls_fail += iw["ls_fail"] + ih["ls_fail"]
        pg = joint_pg(W, Ht)
        rec = dict(i=it, rho_w=rho_w, rho_h=rho_h, pg=pg, w_trace=iw["trace"], h_trace=ih["trace"],
                   f=penalty_objective(A, W, Ht, lam, gamma, L, mode))
        if keep_iterates:
            rec["W"] = W.copy()
            rec["Ht"] = Ht.copy()
        outer.append(rec)
        if pg <= opts.tol * pg0:
            break
    Ad = dense_of(A)
    info = dict(trace=outer, iters=len(outer), pg0=pg0, pg=pg, ls_fail=ls_fail, lam=lam,
                f=penalty_objective(A, W, Ht, lam, gamma, L, mode),
                residual=float(np.linalg.norm(Ad - W @ Ht.T) / np.linalg.norm(Ad)))
    return W, Ht, info
