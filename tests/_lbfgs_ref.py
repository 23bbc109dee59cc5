"""Reference L-BFGS in numpy (test infrastructure): the same algorithm the device solver runs
(Nocedal & Wright Alg. 7.4/7.5 two-loop recursion, step bounded by max_step per coordinate,
Armijo backtracking by halving), driven by the oracle's loss and gradient."""

import numpy as np


def lbfgs(f_and_grad, x0, max_iter, m=10, max_step=1e-3, c1=1e-4, max_backtrack=20):
    x = np.array(x0, dtype=np.float64)
    f, g = f_and_grad(x)
    S, Y = [], []
    trace = [f]
    for _ in range(max_iter):
        if S:
            q = g.copy()
            alphas = []
            for s, y in zip(reversed(S), reversed(Y)):
                a = np.dot(s.ravel(), q.ravel()) / np.dot(y.ravel(), s.ravel())
                alphas.append(a)
                q = q - a * y
            s, y = S[-1], Y[-1]
            r = (np.dot(s.ravel(), y.ravel()) / np.dot(y.ravel(), y.ravel())) * q
            for (s, y), a in zip(zip(S, Y), reversed(alphas)):
                b = np.dot(y.ravel(), r.ravel()) / np.dot(y.ravel(), s.ravel())
                r = r + s * (a - b)
            d = -r
        else:
            d = -g
        gd = np.dot(g.ravel(), d.ravel())
        if not gd < 0:
            S, Y = [], []
            d = -g
            gd = -np.dot(g.ravel(), g.ravel())
        t = min(1.0, max_step / np.max(np.abs(d)))
        for _k in range(max_backtrack + 1):
            xt = x + t * d
            ft, gt = f_and_grad(xt)
            if ft <= f + c1 * t * gd:
                break
            t *= 0.5
        else:
            break
        s, y = xt - x, gt - g
        if np.dot(s.ravel(), y.ravel()) > 0:
            S.append(s)
            Y.append(y)
            if len(S) > m:
                S.pop(0)
                Y.pop(0)
        elif len(S) == m:
            S.pop(0)
            Y.pop(0)
        x, f, g = xt, ft, gt
        trace.append(f)
    return x, trace
