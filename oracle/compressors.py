"""FP64 reference of the compressors of a block (Sec. 4) -- test infrastructure only.

Only the tests and the trials script beside this file use this module; the library never calls
it, and the two share no code. Each routine takes an explicit dense block D (m x n) and sees it
only through the products the paper allows a compressor: a row e_i^T D, a column D e_j, or
products D X and D^T Y with vectors or blocks of vectors. Random numbers are inputs (omega, w1).

  aca(D, eps_stop, kcap, need)
      Algorithm 6 (Sec. 4.1) with partial pivoting: first pivot row 0; the column pivot is the
      entry of largest modulus of the residual row (first on ties); the next pivot row is the
      entry of largest modulus of the new residual column among the rows not used yet; an
      exactly zero residual row is marked used and the first unused row is tried. Stop once
      `need` consecutive crosses meet eq. (truncaca), ||l_r|| ||u_r|| <= eps_stop ||L_{r-1} U_{r-1}||_F
      (the norm of the approximation before the cross, updated from the cross terms), keeping
      every cross; or at min(m, n) or kcap crosses.
  lanczos(D, w1, eps_stop, kcap, need)
      Algorithm 7 (Sec. 4.2), Golub-Kahan-Lanczos bidiagonalization from the unit vector w1, with
      every new q and w orthogonalized twice against all earlier ones. Step r adds
      q_r (alpha_r w_r + beta_r w_{r+1})^T (one step of lookahead), of norm
      sqrt(alpha_r^2 + beta_r^2); stop once `need` consecutive steps meet eq. (truncaca) against
      sum_{s<r} (alpha_s^2 + beta_s^2), or at alpha_r = 0, beta_r = 0, min(m, n) or kcap steps.
  randomized(D, omega, eps, p, rmax)
      Algorithm 8 (Sec. 4.3) in its blocked form: each round samples Y = D Omega_round (the next
      p columns of omega), projects Y twice against the basis Q, orthonormalizes the new columns
      by Gram-Schmidt applied twice and drops a column whose remaining norm is at most
      0.1 eps ||D||_est (||D||_est^2 = ||Y_0||_F^2 / p from the first round); a kept column left
      with less than kappa = 1000 u / eps of its original norm is projected once more against the
      whole basis before it is normalised (Alg. 8 orthogonalises every new sample against all
      earlier ones; at eps = 1e-12 the block form otherwise loses orthogonality), and appends
      W_new = D^T Q_new. It stops when ||W_new||_F <= (eps/2) ||W_old||_F (eq. (truncaca) with the
      block's energy), when no column is kept, when Q has min(m, n) columns, or when the next round
      would pass rmax columns. Returns (Q, W = D^T Q, rounds).
  fixed_rank(D, omega, q)
      Algorithm 9 (Sec. 4.4): L = orth(D Omega) with k = omega's columns, then q times
      U = orth(D^T L), L = orth(D U); finally U = D^T L. Returns (L, U), so D ~ L U^T with rank <= k.
  truncate(L, U, eps)
      Algorithm 5 (Sec. 4): QR of both factors, SVD of the small core, and the eps-rank of the
      core (smallest k with relative Frobenius tail <= eps), giving the best approximation of
      L U^T at relative error eps.

Pins (tests/test_oracle.py): ACA reproduces the pivot rows and columns exactly (its
interpolation property) and a matrix of rank r after r crosses; it skips a zero first row;
Lanczos gives orthonormal Q and W with Q^T D W upper bidiagonal (alpha on the diagonal, beta
above it), and run to full length the singular values of that bidiagonal are those of D (numpy's
SVD); the randomized range finder captures a rank-r matrix exactly in r orthonormal columns,
dropping the rest, and on geometrically decaying singular values its truncated result meets
1.5 eps at rank <= k_eps + 2 (numpy's SVD); the fixed-rank scheme returns rank <= k and, with a
spectral gap after k, comes within 1 % of the best rank-k error (numpy's SVD tail); truncate's
error equals the tail of numpy's singular values of L U^T.
"""
from __future__ import annotations

import numpy as np


def aca(D: np.ndarray, eps_stop: float, kcap: int, need: int = 2):
    """Cross approximation of D: returns (L (m x k), U (n x k), k) with D ~ L U^T."""
    D = np.asarray(D, np.float64)
    m, n = D.shape
    used = np.zeros(m, bool)
    Ls, Us = [], []
    norm2 = 0.0
    hits = 0
    i = 0
    cap = min(m, n, kcap)
    while len(Ls) < cap:
        # residual row i of D - L U^T
        u = D[i, :].copy()
        for l, uu in zip(Ls, Us):
            u -= l[i] * uu
        j = int(np.argmax(np.abs(u)))
        if u[j] == 0.0:
            used[i] = True
            free = np.flatnonzero(~used)
            if free.size == 0:
                break
            i = int(free[0])
            continue
        u = u / u[j]
        # residual column j
        l = D[:, j].copy()
        for ll, uu in zip(Ls, Us):
            l -= uu[j] * ll
        used[i] = True
        cross = sum(float(ll @ l) * float(uu @ u) for ll, uu in zip(Ls, Us))
        prev = norm2
        norm2 = prev + 2.0 * cross + float(l @ l) * float(u @ u)
        Ls.append(l)
        Us.append(u)
        hits = hits + 1 if float(l @ l) * float(u @ u) <= eps_stop * eps_stop * prev else 0
        if hits >= need:
            break
        a = np.abs(l)
        a[used] = -1.0
        if np.all(used):
            break
        i = int(np.argmax(a))
    L = np.array(Ls).T if Ls else np.zeros((m, 0))
    U = np.array(Us).T if Us else np.zeros((n, 0))
    return L, U, len(Ls)


def _orth2(v: np.ndarray, basis) -> np.ndarray:
    """v minus its projection onto the orthonormal vectors in basis, done twice."""
    for _ in range(2):
        for b in basis:
            v = v - float(b @ v) * b
    return v


def lanczos(D: np.ndarray, w1: np.ndarray, eps_stop: float, kcap: int, need: int = 2):
    """Bidiagonalization of D from w1: returns (Q (m x k), W (n x k'), alpha (k), beta (k), k),
    k' = k + 1 when w_{k+1} exists, else k."""
    D = np.asarray(D, np.float64)
    m, n = D.shape
    w = np.asarray(w1, np.float64)
    w = w / np.linalg.norm(w)
    Qs, Ws = [], [w]
    alphas, betas = [], []
    norm2 = 0.0
    hits = 0
    beta = 0.0
    cap = min(m, n, kcap)
    while len(Qs) < cap:
        q = D @ Ws[-1]
        if Qs:
            q = q - beta * Qs[-1]
        q = _orth2(q, Qs)
        alpha = float(np.linalg.norm(q))
        if alpha == 0.0:
            break
        q = q / alpha
        Qs.append(q)
        wn = D.T @ q - alpha * Ws[-1]
        wn = _orth2(wn, Ws)
        beta = float(np.linalg.norm(wn))
        alphas.append(alpha)
        betas.append(beta)
        inc = alpha * alpha + beta * beta
        prev = norm2
        norm2 = prev + inc
        hits = hits + 1 if inc <= eps_stop * eps_stop * prev else 0
        if hits >= need or beta == 0.0 or len(Qs) >= cap:
            break
        Ws.append(wn / beta)
    Q = np.array(Qs).T if Qs else np.zeros((m, 0))
    W = np.array(Ws).T
    return Q, W, np.array(alphas), np.array(betas), len(Qs)


def _gs2_drop(Y: np.ndarray, drop: float) -> np.ndarray:
    """Gram-Schmidt applied twice to the columns of Y in order; a column whose remaining norm is
    at most `drop` is left out. Returns the kept orthonormal columns."""
    kept = []
    for j in range(Y.shape[1]):
        v = _orth2(Y[:, j].copy(), kept)
        nv = float(np.linalg.norm(v))
        if nv > drop:
            kept.append(v / nv)
    return np.array(kept).T if kept else np.zeros((Y.shape[0], 0))


def _gs2_drop_recheck(Y: np.ndarray, drop: float, Q: np.ndarray, ny: np.ndarray, kappa: float) -> np.ndarray:
    """_gs2_drop for the columns of a sample block already projected against the basis Q; a kept
    column left with less than kappa of its original norm ny[j] is projected once more against
    the whole basis (Q and the columns kept before it), since its components along Q, of the
    order of the rounding of ny[j], grow by ny[j] / ||v|| when it is normalised."""
    kept = []
    for j in range(Y.shape[1]):
        v = _orth2(Y[:, j].copy(), kept)
        nv = float(np.linalg.norm(v))
        if drop < nv < kappa * ny[j]:
            B = np.hstack([Q] + ([np.array(kept).T] if kept else []))
            v = v - B @ (B.T @ v)
            nv = float(np.linalg.norm(v))
        if nv > drop:
            kept.append(v / nv)
    return np.array(kept).T if kept else np.zeros((Y.shape[0], 0))


def randomized(D: np.ndarray, omega: np.ndarray, eps: float, p: int, rmax: int):
    """Blocked adaptive range finder of D with the Gaussian columns omega (n x >= rounds * p)."""
    D = np.asarray(D, np.float64)
    m, n = D.shape
    Q = np.zeros((m, 0))
    W = np.zeros((n, 0))
    est = None
    rounds = 0
    while True:
        Om = omega[:, rounds * p:(rounds + 1) * p]
        if Om.shape[1] < p:
            break
        rounds += 1
        Y = D @ Om
        ny = np.linalg.norm(Y, axis=0)
        if est is None:
            est = np.sqrt(float(np.sum(Y * Y)) / p)
        for _ in range(2):
            Y = Y - Q @ (Q.T @ Y)
        Qn = _gs2_drop_recheck(Y, 0.1 * eps * est, Q, ny, 1000.0 * 2.0 ** -53 / eps)
        if Qn.shape[1] == 0:
            break
        Wn = D.T @ Qn
        old2 = float(np.sum(W * W))
        new2 = float(np.sum(Wn * Wn))
        Q = np.hstack([Q, Qn])
        W = np.hstack([W, Wn])
        if new2 <= (0.5 * eps) ** 2 * old2:
            break
        if Q.shape[1] >= min(m, n) or Q.shape[1] + p > rmax:
            break
    return Q, W, rounds


def _orthonormal(Y: np.ndarray) -> np.ndarray:
    return _gs2_drop(Y, 0.0)


def fixed_rank(D: np.ndarray, omega: np.ndarray, q: int):
    """Rank-k approximation L U^T of D (k = omega's columns) with q subspace iterations."""
    D = np.asarray(D, np.float64)
    L = _orthonormal(D @ omega)
    for _ in range(q):
        U = _orthonormal(D.T @ L)
        L = _orthonormal(D @ U)
    return L, D.T @ L


def truncate(L: np.ndarray, U: np.ndarray, eps: float):
    """Best approximation of L U^T at relative Frobenius error eps: (U_k S_k, V_k)."""
    L = np.asarray(L, np.float64)
    U = np.asarray(U, np.float64)
    if L.shape[1] == 0:
        return L.copy(), U.copy()
    QL, RL = np.linalg.qr(L)
    QU, RU = np.linalg.qr(U)
    X, s, Yt = np.linalg.svd(RL @ RU.T)
    tail = np.sqrt(np.cumsum((s * s)[::-1])[::-1])  # tail[k] = ||s[k:]||
    total = tail[0]
    k = 0
    while k < len(s) and tail[k] > eps * total:
        k += 1
    return QL @ (X[:, :k] * s[:k]), QU @ Yt[:k, :].T
