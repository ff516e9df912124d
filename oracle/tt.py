"""Tensor-train arithmetic (oracle; test infrastructure only).

A TT is a list of complex float64 cores C_k of shape (r_{k-1}, n, r_k) with
r_0 = r_d = 1 (App. A, "Tensor train decomposition").  Flattenings follow the
paper's column-major convention C[i,j,k] = v[i + a j + a b k]:
H(C) = C.reshape(a, b c, order="F") (horizontal) and
V(C) = C.reshape(a b, c, order="F") (vertical).

The rounding takes the direction the solver uses: the orthogonalisation is
Alg. 1 mirrored (right-to-left, LQ factorisations, the paper's "Right-to-Left
orthogonalization"), and the truncation is Alg. 2 mirrored (left-to-right
truncated SVDs with per-SVD tolerance eps/sqrt(d-1)).
"""
from __future__ import annotations

import numpy as np


def H(C):
    a, b, c = C.shape
    return C.reshape(a, b * c, order="F")


def V(C):
    a, b, c = C.shape
    return C.reshape(a * b, c, order="F")


def unH(M, a, b, c):
    return np.asfortranarray(np.asarray(M).reshape(a, b, c, order="F"))


def unV(M, a, b, c):
    return np.asfortranarray(np.asarray(M).reshape(a, b, c, order="F"))


def ranks(cores):
    return [1] + [c.shape[2] for c in cores]


def full(cores):
    """Full tensor f[i_1..i_d] = C_1[1,i_1,:] C_2[:,i_2,:] ... C_d[:,i_d,1]
    (the iterated matrix product that defines the format)."""
    d = len(cores)
    n = [c.shape[1] for c in cores]
    cur = cores[0].reshape(n[0], cores[0].shape[2])  # (i_1, r_1)
    for k in range(1, d):
        a, b, c = cores[k].shape
        cur = np.tensordot(cur, cores[k], axes=([cur.ndim - 1], [0]))
    return cur.reshape(n)


def evaluate(cores, idx):
    """Entries at integer multi-indices idx (npts x d) by the iterated matrix
    product, one point at a time."""
    idx = np.asarray(idx)
    out = np.empty(idx.shape[0], dtype=complex)
    for p in range(idx.shape[0]):
        v = np.ones((1,), dtype=complex)
        for k, C in enumerate(cores):
            v = v @ C[:, idx[p, k], :]
        out[p] = v[0]
    return out


def tt_sum(terms):
    """sum_t coef_t * f_t by block concatenation: first cores side by side,
    interior cores block diagonal, last cores stacked (App. A, the TT sum;
    the scalar goes into the first core, App. A scalar multiplication).
    ``terms`` is a list of (coef, cores)."""
    d = len(terms[0][1])
    out = []
    for k in range(d):
        blocks = [c[k] for _, c in terms]
        if k == 0:
            core = np.concatenate([coef * b for (coef, _), b in zip(terms, blocks)], axis=2)
        elif k == d - 1:
            core = np.concatenate(blocks, axis=0)
        else:
            a = sum(b.shape[0] for b in blocks)
            c = sum(b.shape[2] for b in blocks)
            n = blocks[0].shape[1]
            core = np.zeros((a, n, c), dtype=complex)
            ia = ic = 0
            for b in blocks:
                core[ia:ia + b.shape[0], :, ic:ic + b.shape[2]] = b
                ia += b.shape[0]
                ic += b.shape[2]
        out.append(np.asfortranarray(core))
    return out


def scale(cores, alpha):
    out = [c.copy() for c in cores]
    out[0] = out[0] * alpha
    return out


def apply_mpo(cores, W, bond):
    """Y = G X core by core: Y_k[(alpha, i), m, (beta, j)] =
    sum_m' W_k[alpha,beta][m, m'] X_k[i, m', j], with the combined rank index
    alpha * r + i (block alpha holds a contiguous run of r indices).  Output
    ranks are 6 r (interior).  Pinned against fullgrid.apply_G."""
    d = len(cores)
    out = []
    for k in range(d):
        X = cores[k]
        a, n, c = X.shape
        Al, Ar = bond[k], bond[k + 1]
        Y = np.zeros((Al * a, n, Ar * c), dtype=complex)
        for (al, be), M in W[k].items():
            Y[al * a:(al + 1) * a, :, be * c:(be + 1) * c] = np.einsum("mp,ipj->imj", M, X)
        out.append(np.asfortranarray(Y))
    return out


def orthogonalize_rl(cores):
    """Right-to-left orthogonalisation (Alg. 1 mirrored with LQ factors):
    for c = d..2, H(Y_c) = L_c Q_c, Y_c <- Q_c, V(Y_{c-1}) <- V(Y_{c-1}) L_c.
    Afterwards H(Y_c) H(Y_c)^H = I for c >= 2 and the norm sits in Y_1."""
    Y = [c.copy() for c in cores]
    d = len(Y)
    for c in range(d - 1, 0, -1):
        a, b, cc = Y[c].shape
        Qt, Rt = np.linalg.qr(H(Y[c]).conj().T)  # H^H = Qt Rt  <=>  H = Rt^H Qt^H
        L = Rt.conj().T
        Q = Qt.conj().T
        p = Q.shape[0]
        Y[c] = unH(Q, p, b, cc)
        a2, b2, _ = Y[c - 1].shape
        Y[c - 1] = unV(V(Y[c - 1]) @ L, a2, b2, p)
    return Y


def choose_rank(s, eps_hat, cap):
    """Smallest rho >= 1 with sqrt(sum_{i >= rho} s_i^2) <= eps_hat, then
    min(rho, cap).  Returns (rho, discarded norm at rho)."""
    s = np.asarray(s, dtype=float)
    tail2 = np.concatenate([np.cumsum((s[::-1]) ** 2)[::-1], [0.0]])  # tail2[r] = sum s[r:]^2
    rho = len(s)
    for r in range(1, len(s) + 1):
        if np.sqrt(tail2[r]) <= eps_hat:
            rho = r
            break
    rho = max(1, min(rho, cap))
    return rho, float(np.sqrt(tail2[rho]))


def round_tt(cores, tol, cap, forced_ranks=None):
    """TT rounding (Alg. 2, mirrored): orthogonalise right-to-left, take
    ||f|| = ||Y_1||_F, eps = tol ||f||, eps_hat = eps / sqrt(d-1); then for
    c = 1..d-1 the truncated SVD of V(Z_c) = U S V^H keeps rho columns,
    Z_c <- U_rho and H(Z_{c+1}) <- S_rho V_rho^H H(Z_{c+1}).
    ``forced_ranks`` (length d+1) replays given ranks instead of choosing.
    Returns (cores, ranks, discarded) with discarded = sqrt(sum delta_c^2),
    the bound on ||g - f|| (Alg. 2 result statement)."""
    d = len(cores)
    if d < 2:
        return [c.copy() for c in cores], ranks(cores), 0.0
    Y = orthogonalize_rl(cores)
    nrm = float(np.linalg.norm(Y[0]))
    eps_hat = tol * nrm / np.sqrt(d - 1)
    disc2 = 0.0
    for c in range(d - 1):
        a, b, cc = Y[c].shape
        U, s, Vh = np.linalg.svd(V(Y[c]), full_matrices=False)
        if forced_ranks is not None:
            rho = int(forced_ranks[c + 1])
            if not (1 <= rho <= len(s)):
                raise ValueError("forced rank out of range")
            delta = float(np.sqrt(np.sum(s[rho:] ** 2)))
        else:
            rho, delta = choose_rank(s, eps_hat, cap)
        disc2 += delta ** 2
        Y[c] = unV(U[:, :rho], a, b, rho)
        SV = s[:rho, None] * Vh[:rho]
        a3, b3, c3 = Y[c + 1].shape
        Y[c + 1] = unH(SV @ H(Y[c + 1]), rho, b3, c3)
    return Y, ranks(Y), float(np.sqrt(disc2))


def norm(cores):
    """||f||_F by orthogonalisation (stable; norm of the first core after the
    right-to-left sweep)."""
    return float(np.linalg.norm(orthogonalize_rl(cores)[0]))


def diff_norm(x, y):
    """||x - y||_F via the TT of x - y (block sum), orthogonalised."""
    return norm(tt_sum([(1.0, x), (-1.0, y)]))


def tt_svd(F, tol, cap):
    """TT-SVD of a full tensor (sequential truncated SVDs of unfoldings,
    per-SVD tolerance tol ||F|| / sqrt(d-1), cap on every rank)."""
    d = F.ndim
    n = F.shape
    eps_hat = tol * np.linalg.norm(F) / np.sqrt(max(d - 1, 1))
    cores = []
    r = 1
    M = F.reshape(n[0], -1, order="F")
    for k in range(d - 1):
        M = M.reshape(r * n[k], -1, order="F")
        U, s, Vh = np.linalg.svd(M, full_matrices=False)
        rho, _ = choose_rank(s, eps_hat, cap)
        cores.append(unV(U[:, :rho], r, n[k], rho))
        M = s[:rho, None] * Vh[:rho]
        r = rho
    cores.append(unH(M.reshape(r, n[d - 1], order="F"), r, n[d - 1], 1))
    return cores


def rk4_step(cores, dt, W, bond, tol, cap, replay=None, record=None):
    """One step-truncation RK4 step (Eq. discrete-flow-trunc-intro with the
    classical RK4 increment): K_s = T[G Y_s], Y_2 = T[f + dt/2 K_1],
    Y_3 = T[f + dt/2 K_2], Y_4 = T[f + dt K_3], f_new = T[f + dt/6 (K_1 + 2K_2
    + 2K_3 + K_4)].  Every T is ``round_tt`` at (tol, cap).  ``replay`` is an
    iterator of forced rank lists (one per rounding, 8 per step), ``record``
    a list that receives the chosen rank lists.  Returns (cores, discarded
    norms of the 8 roundings)."""
    discs = []

    def T(x):
        forced = next(replay) if replay is not None else None
        y, r, disc = round_tt(x, tol, cap, forced)
        if record is not None:
            record.append(r)
        discs.append(disc)
        return y

    G = lambda x: apply_mpo(x, W, bond)
    f = cores
    K1 = T(G(f))
    Y2 = T(tt_sum([(1.0, f), (0.5 * dt, K1)]))
    K2 = T(G(Y2))
    Y3 = T(tt_sum([(1.0, f), (0.5 * dt, K2)]))
    K3 = T(G(Y3))
    Y4 = T(tt_sum([(1.0, f), (dt, K3)]))
    K4 = T(G(Y4))
    fn = T(tt_sum([(1.0, f), (dt / 6, K1), (dt / 3, K2), (dt / 3, K3), (dt / 6, K4)]))
    return fn, discs


def moments(cores, n, L, da):
    """Mean and covariance of u_bar from central differences at a = 0 (same
    formulas as fullgrid.moments), contracted core by core: each core is
    reduced at indices c-1, c, c+1 (c = n/2) and left/right environment
    products give every first and mixed second difference."""
    d = len(cores)
    c = n // 2
    E0 = [C[:, c, :] for C in cores]
    Ep = [C[:, c + 1, :] for C in cores]
    Em = [C[:, c - 1, :] for C in cores]

    def chain(mats):
        v = np.ones((1, 1), dtype=complex)
        for M in mats:
            v = v @ M
        return v[0, 0]

    def at(offsets):
        mats = list(E0)
        for ax, o in offsets:
            mats[ax] = Ep[ax] if o > 0 else Em[ax]
        return chain(mats)

    mean = np.zeros(d)
    second = np.zeros((d, d))
    phi0 = at([])
    for k in range(d):
        mean[k] = (-1j * (at([(k, 1)]) - at([(k, -1)])) / (2 * da)).real
    for j in range(d):
        for k in range(d):
            if j == k:
                v = -(at([(k, 1)]) - 2 * phi0 + at([(k, -1)])) / da ** 2
            else:
                v = -(at([(j, 1), (k, 1)]) - at([(j, 1), (k, -1)])
                      - at([(j, -1), (k, 1)]) + at([(j, -1), (k, -1)])) / (4 * da ** 2)
            second[j, k] = v.real
    return mean, second - np.outer(mean, mean)


def euler_step(cores, dt, G, tol, cap, replay=None, record=None):
    """Truncated explicit Euler (Eq. adaptive-euler-method):
    f_{k+1} = T_r[f_k + dt T_s[G(f_k)]], both truncations ``round_tt`` at
    (tol, cap).  ``G`` applies the operator to a TT (e.g. apply_mpo with the
    operator's blocks); replay/record as in rk4_step.  Returns (cores,
    discarded norms of the 2 roundings)."""
    discs = []

    def T(x):
        forced = next(replay) if replay is not None else None
        y, r, disc = round_tt(x, tol, cap, forced)
        if record is not None:
            record.append(r)
        discs.append(disc)
        return y

    K = T(G(cores))
    return T(tt_sum([(1.0, cores), (dt, K)])), discs


def midpoint_step(cores, dt, G, tol, cap, replay=None, record=None):
    """Truncated explicit midpoint (Eq. adaptive-midpoint-method):
    f_{k+1} = T_a[f_k + dt T_b[G(f_k + dt/2 T_c(G(f_k)))]]; the inner sum
    f_k + dt/2 T_c(G f_k) is not truncated, as printed.  Returns (cores,
    discarded norms of the 3 roundings)."""
    discs = []

    def T(x):
        forced = next(replay) if replay is not None else None
        y, r, disc = round_tt(x, tol, cap, forced)
        if record is not None:
            record.append(r)
        discs.append(disc)
        return y

    K1 = T(G(cores))
    Y = tt_sum([(1.0, cores), (0.5 * dt, K1)])
    K2 = T(G(Y))
    return T(tt_sum([(1.0, cores), (dt, K2)])), discs
