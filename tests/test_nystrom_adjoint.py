"""The reverse pass's stage sweep in Nystrom form (CPU): for second-order systems y = (x, v),
f = (v, a(x)), the FP32 kernels carry only the accelerations' cotangents abar_j. Seeded from the new
state's cotangent by h b_j ybar_v + h^2 (bA)_j ybar_x (with ybar_v += h ybar_x), and from a dense
output's by h wd_j w_v + h^2 (wd A)_j w_x (with ybar_v += h (sum_j wd_j) w_x), the sweep
Xbar_j = J_a^T abar_j, ybar_x += Xbar_j, ybar_v += h c'_j Xbar_j, abar_l += h^2 (A^2)_jl Xbar_j gives
the general sweep's gradient (kbar_l += h a_jl J_f^T kbar_j over six components), which is the
gradient of the step. Written out here for a linear acceleration, on the oracle's tableaux."""
import numpy as np

import oracle as O


def _step(A, b, wd, M, h, y):
    S = len(b)
    K = np.zeros((S, 6))
    for j in range(S):
        Yj = y + h * (A[j, :j] @ K[:j])
        K[j] = np.concatenate([Yj[3:], M @ Yj[:3]])
    return y + h * (b @ K), y + h * (wd @ K)


def test_nystrom_sweep_equals_the_general_sweep_and_the_gradient():
    rng = np.random.default_rng(1)
    for method in ("tsit5", "dopri5"):
        T = O.tableau(method)
        A, b = np.array(T["A"]), np.array(T["b"])
        S = T["s"]
        M = rng.normal(size=(3, 3))
        M = M + M.T
        h, wd = 0.3, rng.normal(size=S)
        g1, g2, y0 = rng.normal(size=6), rng.normal(size=6), rng.normal(size=6)
        loss = lambda y: g1 @ _step(A, b, wd, M, h, y)[0] + g2 @ _step(A, b, wd, M, h, y)[1]
        fd = np.array([(loss(y0 + 1e-6 * e) - loss(y0 - 1e-6 * e)) / 2e-6 for e in np.eye(6)])
        # general sweep
        kbar = h * wd[:, None] * g2[None, :] + h * b[:, None] * g1[None, :]
        ybar = g1 + g2
        for j in range(S - 1, -1, -1):
            gy = np.concatenate([M.T @ kbar[j][3:], kbar[j][:3]])
            ybar = ybar + gy
            for l in range(j):
                kbar[l] += h * A[j, l] * gy
        general = ybar
        # Nystrom sweep
        AA, c = A @ A, A.sum(1)
        ab = h * wd[:, None] * g2[None, 3:] + h * h * (wd @ A)[:, None] * g2[None, :3]
        ab += h * b[:, None] * g1[None, 3:] + h * h * (b @ A)[:, None] * g1[None, :3]
        ybar = g1.copy()
        ybar[3:] += h * ybar[:3]
        ybar[:3] += g2[:3]
        ybar[3:] += g2[3:] + h * wd.sum() * g2[:3]
        for j in range(S - 1, -1, -1):
            X = M.T @ ab[j]
            ybar[:3] += X
            ybar[3:] += h * c[j] * X
            for l in range(j - 1):
                ab[l] += h * h * AA[j, l] * X
        assert np.abs(general - fd).max() < 1e-8
        assert np.abs(ybar - general).max() < 1e-13
