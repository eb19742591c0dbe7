"""Preconditioned conjugate gradients (oracle; test infrastructure).

Section 6 uses a low-accuracy TLR Cholesky factorization (of A + eps I) as the
preconditioner of CG and counts the iterations needed to reach
||A x - b|| / ||b|| <= tol, with at most 300 iterations.  This is the textbook
preconditioned CG (Saad, Iterative Methods for Sparse Linear Systems, 2nd ed.,
Algorithm 9.1), one right-hand side at a time, started from x = 0, stopped on
the recursively updated residual; the true residual of the result is reported
beside it.
"""
import numpy as np


def pcg(apply_A, apply_Minv, b, tol: float, maxit: int):
    """Solve A x = b for each column of b; return (x, iterations, true relative residual) per column.

    apply_A(X) and apply_Minv(R) act on N x k arrays.  A zero column converges at 0 iterations with x = 0.
    """
    b = np.asarray(b, dtype=np.float64).reshape(b.shape[0], -1)
    n, k = b.shape
    x = np.zeros((n, k))
    iters = np.zeros(k, dtype=np.int64)
    for c in range(k):
        bc = b[:, c:c + 1]
        bn = np.linalg.norm(bc)
        if bn == 0.0:
            continue
        xc = np.zeros((n, 1))
        r = bc.copy()
        z = apply_Minv(r)
        p = z.copy()
        rz = float(r[:, 0] @ z[:, 0])
        it = 0
        while it < maxit:
            it += 1
            q = apply_A(p)
            alpha = rz / float(p[:, 0] @ q[:, 0])
            xc = xc + alpha * p
            r = r - alpha * q
            if np.linalg.norm(r) <= tol * bn:
                break
            z = apply_Minv(r)
            rz_new = float(r[:, 0] @ z[:, 0])
            p = z + (rz_new / rz) * p
            rz = rz_new
        x[:, c] = xc[:, 0]
        iters[c] = it
    res = np.zeros(k)
    ax = apply_A(x)
    for c in range(k):
        bn = np.linalg.norm(b[:, c])
        res[c] = np.linalg.norm(b[:, c] - ax[:, c]) / bn if bn > 0 else 0.0
    return x, iters, res
