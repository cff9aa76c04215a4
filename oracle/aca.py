"""Partially pivoted adaptive cross approximation with QR/SVD recompression
(Eq. 11-12: Z_sub ~ A B with ||Z_sub - A B||_F <= eps ||Z_sub||_F; the
"re-compressed ACA" of Sec. II).

Reading (the paper names the method, not its variant):
  * the first pivot row is local row 0;
  * each step takes the residual row i, its pivot column j = argmax |row|,
    v = row / row[j], the residual column j as u, so that block ~ sum u v^T;
  * the Frobenius norm of the approximation is updated incrementally,
      ||S_k||^2 = ||S_k-1||^2 + 2 Re sum_l (u_l^H u_k) conj(v_l^H v_k) + |u_k|^2 |v_k|^2;
  * stop when |u_k| |v_k| <= eps ||S_k||_F or when no row is left;
  * next row = argmax |u_k| over unused rows (lowest index on ties); a row
    whose residual is exactly zero is marked used and the lowest unused row
    is tried next;
  * recompression: U = Q_U R_U, V = Q_V R_V, R_U R_V^T = W S Y^H, keep the
    singular values >= eps * s_1; U' = Q_U W S, V' = Q_V conj(Y);
  * a block whose recompressed rank r has r (m + n) >= m n is kept dense.

Pinned by: ||Z_blk - U V^T||_F <= eps ||Z_blk||_F against the directly filled
block (with a small safety factor for the heuristic stopping rule), exact
recovery of an explicitly rank-r matrix, and rank 0 for a zero block.
"""
import numpy as np


def aca(row_fn, col_fn, m, n, eps, max_rank=None):
    """row_fn(i) -> (n,) complex row of the block; col_fn(j) -> (m,) column.

    Returns U (m, r), V (n, r) with block ~ U V^T."""
    if max_rank is None:
        max_rank = min(m, n)
    us, vs = [], []
    used = np.zeros(m, dtype=bool)
    norm2 = 0.0
    i = 0
    while len(us) < max_rank:
        used[i] = True
        row = row_fn(i).astype(np.complex128)
        for u, v in zip(us, vs):
            row -= u[i] * v
        j = int(np.argmax(np.abs(row)))
        if row[j] == 0.0:
            free = np.flatnonzero(~used)
            if len(free) == 0:
                break
            i = int(free[0])
            continue
        v = row / row[j]
        u = col_fn(j).astype(np.complex128)
        for uu, vv in zip(us, vs):
            u -= vv[j] * uu
        nu2 = float(np.vdot(u, u).real)
        nv2 = float(np.vdot(v, v).real)
        cross = 0.0
        for uu, vv in zip(us, vs):
            cross += 2.0 * (np.vdot(uu, u) * np.conj(np.vdot(vv, v))).real
        norm2 = norm2 + cross + nu2 * nv2
        us.append(u)
        vs.append(v)
        if np.sqrt(nu2 * nv2) <= eps * np.sqrt(max(norm2, 0.0)):
            break
        cand = np.abs(u)
        cand[used] = -1.0
        if cand.max() < 0.0:
            break
        i = int(np.argmax(cand))
    if not us:
        return np.zeros((m, 0), np.complex128), np.zeros((n, 0), np.complex128)
    return np.stack(us, axis=1), np.stack(vs, axis=1)


def recompress(U, V, eps):
    """QR of both factors, SVD of the small core, truncation at eps * s_1."""
    r = U.shape[1]
    if r == 0:
        return U, V
    Qu, Ru = np.linalg.qr(U)
    Qv, Rv = np.linalg.qr(V)
    W, s, Yh = np.linalg.svd(Ru @ Rv.T)
    keep = int(np.sum(s >= eps * s[0])) if s[0] > 0 else 0
    U2 = Qu @ (W[:, :keep] * s[:keep][None, :])
    V2 = Qv @ Yh[:keep, :].T            # = Q_V conj(Y[:, :keep])
    return U2, V2
