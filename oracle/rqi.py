"""Multigrid setup and Rayleigh quotient iteration (Algorithm 1), FP64 oracle.

Setup (Sec. 2.1, the paragraph after Algorithm 1): a few smoother iterations
on random vectors give the first test vectors and P; then, a few times, one
multigrid iteration is applied to every test vector, the test vectors are
orthonormalised again and P and the coarse operator are rebuilt (the setup's
coarse solves run without deflation: its test vectors are no eigenvector
approximations yet).  The smoother
iterations on a random w approximate Q^-1 w (SAP: D x = gamma5 w from x = 0);
one multigrid iteration on w is w <- B w with B the two-grid preconditioner at
sigma = 0.

Before the iteration the test vectors are rotated to the Ritz vectors of Q in
their span and ordered by |theta| (same span, hence the same P); N_eig + N_guard
start vectors v_i of Algorithm 1 follow (beyond N_tv: extra_start_vectors), and
the N_eig pairs of smallest |lambda| are returned.  The guard vectors
(N_guard = max(N_eig, N_tv) by default) lower the chance of missing a wanted
pair, the failure the paper describes after Algorithm 1, by spanning whole
clusters of nearly equal eigenvalues.

With ritz_start off the test vectors start Algorithm 1 in the setup's order;
with adaptive_tol off every shifted solve runs to solve_tol.  With every
addition off (ritz_start, adaptive_tol, ritz_each_sweep, fine_deflate,
coarse_deflate, shift_floor = 0, n_guard = 0) this is Algorithm 1 in the
paper's order.

Algorithm 1, per sweep over the unconverged i:
    sigma   = lambda_i * max(1 - max(eps_i, floor), 0)     (damped shift; floor:
              shift_floor, so that |lambda - sigma| stays resolvable)
    v_i    <- (Q - sigma)^-1 v_i                           (FGMRES + two-grid, FP64, to
              relative residual min(solve_tol, 0.1 eps / |lambda_i - sigma|) with
              adaptive_tol, else solve_tol: the new vector's eigen-residual is
              about that tolerance times |lambda_i - sigma|;
              with fine_deflate the two-grid preconditioner is deflated by v_i and
              the iterated vectors whose Rayleigh quotient lies within
              fine_deflate_radius of sigma, see deflated_preconditioner)
    v_i    <- v_i - sum_{j<i} <v_j|v_i> v_j                 (classical GS, done twice)
    v_i    <- v_i / ||v_i||
    update v_i in P (rebuild P and the coarse operator)
    lambda_i = <v_i|Q|v_i>,  eps_i = ||Q v_i - lambda_i v_i||
starting from lambda_i = 0, eps_i = 1.  P is built from the first N_tv of
[v_1, v_2, ...] followed by the remaining test vectors when fewer vectors are
iterated than there are test vectors; updating a v_i beyond the first N_tv leaves P
unchanged.

After every sweep (with ritz_each_sweep) converged pairs are locked, nearly
converged ones (eps_i <= ritz_keep) are only orthonormalised against them, and
the others are replaced by the Ritz vectors of Q in their span (orthogonal to
both); all vectors are kept in |lambda| order.  Vector-wise RQI has no
view of a cluster of nearly equal eigenvalues; the projection separates the
vectors inside one, and locking keeps a converged pair from being mixed again
with inaccurate neighbours.
"""
from __future__ import annotations

import numpy as np

from . import dirac, krylov, mg


def orthonormalise(W: np.ndarray) -> np.ndarray:
    """Gram-Schmidt (each step twice) of the vectors W[0], W[1], ..."""
    out = []
    for w in W:
        w = w.copy()
        for _ in range(2):
            for v in out:
                w = w - np.vdot(v, w) * v
        out.append(w / dirac.norm(w))
    return np.array(out)


def setup(op: dirac.WilsonClover, W0: np.ndarray, params: dict):
    """Test vectors after the setup; returns (W, two-grid preconditioner)."""
    p = params
    W = []
    if p["smoother"] == "sap":
        sap = mg.SAP(op, p["sap_block"])
        for w in W0:
            W.append(sap.smooth(dirac.gamma5(w), np.zeros_like(w), 0.0, p["setup_smooth"], p["sap_mr_iters"]))
    else:
        for w in W0:
            x, _ = krylov.gmres(op.Q, w, tol=0.0, restart=p["gmres_smooth_k"],
                                maxiter=p["gmres_smooth_k"] * p["setup_smooth"])
            W.append(x)
    W = orthonormalise(np.array(W))
    B = mg.TwoGrid(op, W, p)
    B.deflate_active = False
    for _ in range(p["setup_iters"]):
        W = orthonormalise(np.array([B(w, 0.0) for w in W]))
        B.set_test_vectors(W)
    B.deflate_active = True
    return W, B


def ritz_rotate(op: dirac.WilsonClover, W: np.ndarray):
    """Ritz vectors of Q in span(W), ordered by |theta| then theta."""
    QW = np.array([op.Q(w) for w in W])
    n = W.shape[0]
    H = np.einsum("ia,ja->ij", np.conj(W.reshape(n, -1)), QW.reshape(n, -1))
    H = 0.5 * (H + H.conj().T)
    th, Y = np.linalg.eigh(H)
    order = np.lexsort((th, np.abs(th)))
    th, Y = th[order], Y[:, order]
    return np.einsum("ij,i...->j...", Y, W), th


def rayleigh(op: dirac.WilsonClover, v: np.ndarray):
    Qv = op.Q(v)
    lam = float(np.real(np.vdot(v, Qv)))
    return lam, dirac.norm(Qv - lam * v)


def deflated_preconditioner(op: dirac.WilsonClover, Z: np.ndarray, B: mg.TwoGrid, sigma: float):
    """Two-grid preconditioner deflated by the iterated vectors Z (fine_deflate):
        z = Z E^-1 Z^dag r + B (r - (Q - sigma) Z E^-1 Z^dag r),  E = Z^dag (Q - sigma) Z.
    span(Z) is solved exactly (a Galerkin projection); the system solved by
    FGMRES, (Q - sigma) x = v, is unchanged."""
    shape = Z.shape[1:]
    Zf = Z.reshape(len(Z), -1)
    AZ = np.array([op.Q_sigma(z, sigma) for z in Z]).reshape(len(Z), -1)
    E = Zf.conj() @ AZ.T                      # E_jl = <z_j, (Q - sigma) z_l>
    Einv = np.linalg.inv(E)

    def apply(r):
        d = Einv @ (Zf.conj() @ r.reshape(-1))
        rd = (r.reshape(-1) - AZ.T @ d).reshape(shape)
        return (Zf.T @ d).reshape(shape) + B(rd, sigma)
    return apply


def rqi(op: dirac.WilsonClover, V: np.ndarray, extra: np.ndarray, B: mg.TwoGrid,
        n_eig: int, eps: float, params: dict, max_sweeps: int = 50, log=None, n_want: int = None):
    """Algorithm 1.  Returns (lambda, vectors, eps_i, stats), sorted by |lambda|.

    With ritz_each_sweep: pairs with eps_i <= eps are locked (frozen); after every
    sweep the unlocked vectors are orthonormalised against the locked ones and
    replaced by the Ritz vectors of Q in their span, all vectors are kept in
    |lambda| order, and the iteration stops once the n_want lowest are locked
    (the others only widen the span).  Without it, all n_eig must converge."""
    p = params
    ritz_each_sweep = p.get("ritz_each_sweep", True)
    n_want = n_eig if n_want is None else n_want
    V = [v.copy() for v in V[:n_eig]]
    lam = np.zeros(n_eig)
    res = np.ones(n_eig)
    stats = dict(sweeps=0, solves=0, outer_iters=0)
    ntv = B.P.ntv

    def rebuild():
        W = np.array(V + ([] if extra is None else list(extra)))[:ntv]
        B.set_test_vectors(W)

    def unconverged():
        return np.any(res[:n_want] > eps) if ritz_each_sweep else np.any(res > eps)

    rebuild()
    while unconverged() and stats["sweeps"] < max_sweeps:
        stats["sweeps"] += 1
        locked = res <= eps
        for i in range(n_eig):
            if res[i] <= eps:
                continue
            # damped shift, with a floor on the damping (keeps the shifted system
            # solvable by a single precision preconditioner)
            sigma = lam[i] * max(1.0 - max(res[i], p.get("shift_floor", 0.0)), 0.0)
            guard = ritz_each_sweep and i >= n_want
            maxit = min(p.get("guard_maxiter", 4), p["outer_maxiter"]) if guard else p["outer_maxiter"]
            # inexact solve: the new vector's eigen-residual is about tau |lambda - sigma|
            dls = abs(lam[i] - sigma)
            if guard or dls == 0 or not p.get("adaptive_tol", True):
                tau = p["solve_tol"]
            else:
                tau = min(p["solve_tol"], max(0.1 * eps / dls, 1e-12))
            if p.get("fine_deflate", False):
                # z_i and the iterated vectors with Rayleigh quotient within the radius of sigma
                rad = p.get("fine_deflate_radius", -1.0)
                theta = [np.real(np.vdot(v, op.Q(v))) / np.real(np.vdot(v, v)) for v in V]
                S = [i] + [j for j in range(n_eig) if j != i and (rad < 0 or abs(theta[j] - sigma) <= rad)]
                precond = deflated_preconditioner(op, np.array([V[j] for j in S]), B, sigma)
            else:
                precond = lambda r: B(r, sigma)
            x, info = krylov.fgmres(lambda v: op.Q_sigma(v, sigma), precond, V[i],
                                    tol=tau, restart=p["outer_restart"], maxiter=maxit)
            stats["solves"] += 1
            stats["outer_iters"] += info["iters"]
            # Gram-Schmidt against v_j, j < i (Algorithm 1) and every locked pair
            others = [j for j in range(n_eig) if j < i or (ritz_each_sweep and locked[j] and j != i)]
            for _ in range(2):
                coeff = [np.vdot(V[j], x) for j in others]
                for c, j in zip(coeff, others):
                    x = x - c * V[j]
            V[i] = x / dirac.norm(x)
            if i < ntv:
                rebuild()
            lam[i], res[i] = rayleigh(op, V[i])
            if log is not None:
                log(f"sweep {stats['sweeps']} i={i} sigma={sigma:.6e} lambda={lam[i]:.12e} eps={res[i]:.3e} "
                    f"outer={info['iters']}")
        if ritz_each_sweep:
            keep = p.get("ritz_keep", 0.0)
            L = [i for i in range(n_eig) if res[i] <= eps]
            K = [i for i in range(n_eig) if eps < res[i] <= keep]
            Uo = [i for i in range(n_eig) if res[i] > max(eps, keep)]
            if K or Uo:
                X = orthonormalise(np.array([V[i] for i in L + K + Uo]))[len(L):]
                R = X[len(K):]
                if Uo:
                    R, _ = ritz_rotate(op, R)
                for k, i in enumerate(K + Uo):
                    V[i] = X[k] if k < len(K) else R[k - len(K)]
                    lam[i], res[i] = rayleigh(op, V[i])
            order = list(np.lexsort((lam, np.abs(lam))))
            V = [V[k] for k in order]
            lam, res = lam[order], res[order]
            rebuild()
    order = np.lexsort((lam, np.abs(lam)))
    return lam[order], np.array(V)[order], res[order], stats


def extra_start_vectors(op: dirac.WilsonClover, B: mg.TwoGrid, W: np.ndarray, n: int, seed: int, params: dict):
    """n further start vectors for Algorithm 1 beyond the N_tv test vectors:
    Philox uniforms (tag TAG_EXTRA), setup_smooth two-grid iterations at sigma = 0
    with the setup's P, orthonormalised against W and each other."""
    import synth
    X = synth.uniform_vectors(op.dims, n, seed, tag=synth.TAG_EXTRA)
    B.deflate_active = False
    for _ in range(params["setup_smooth"]):
        X = np.array([B(x, 0.0) for x in X])
    B.deflate_active = True
    return orthonormalise(np.concatenate([W, X]))[len(W):]


def eigensolve(op: dirac.WilsonClover, W0: np.ndarray, n_eig: int, eps: float, params: dict,
               max_sweeps: int = 50, log=None, n_guard: int = -1, seed: int = 0):
    """Setup, Ritz rotation of the test vectors, then Algorithm 1 on n_eig + n_guard
    vectors.  Vectors beyond the N_tv test vectors come from extra_start_vectors;
    P is always built from the N_tv iterated vectors of smallest |theta| (in the
    Ritz order) plus, when N_tv exceeds the number iterated, the remaining test vectors."""
    W, B = setup(op, W0, params)
    ntv = W.shape[0]
    guard = max(n_eig, ntv) if n_guard < 0 else n_guard
    n_run = n_eig + guard
    if n_run > ntv:
        W = np.concatenate([W, extra_start_vectors(op, B, W, n_run - ntv, seed, params)])
    if params.get("ritz_start", True):
        W, _ = ritz_rotate(op, W)
    extra = W[n_run:] if W.shape[0] > n_run else None
    lam, V, res, st = rqi(op, W[:n_run], extra, B, n_run, eps, params, max_sweeps, log, n_want=n_eig)
    return lam[:n_eig], V[:n_eig], res[:n_eig], st
