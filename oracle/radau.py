"""Adaptive Radau IIA collocation for the linear system dc/dt = A(t) c.

Test infrastructure (see ``oracle/__init__``).

The paper integrates its semi-discrete system "with a multistep integrator"
(Section 2.1, last paragraph) without naming a tolerance; the oracle instead
defines its reference result as the converged solution of the Galerkin ODE,
obtained with an L-stable collocation method at a tight tolerance.

* Coefficients come from the collocation definition, not from a printed
  tableau: the nodes are the zeros of d^{s-1}/dx^{s-1} [x^{s-1} (x-1)^s]
  (right Radau points on [0, 1]); a_ij = integral_0^{c_i} l_j(x) dx with l_j
  the Lagrange basis on the nodes; b = last row of a.
* Each step solves the full linear stage system
      Y_i = c_n + h sum_j a_ij A(t_n + c_j h) Y_j,  i = 1..s
  directly (dense LU); the new state is Y_s (stiffly accurate).
* Step-size control by step doubling: one step of h against two of h/2; the
  difference (an estimate of the error of the single step, hence a bound on
  the kept two-step result) must not exceed atol + rtol*|c|_inf in the max norm.
* Sample times are hit exactly (a step never crosses the next output time).

Parity status: pinned (order conditions of the tableau, convergence order on
a scalar test equation with a closed form, self-convergence in rtol).
"""
import numpy as np
from numpy.polynomial import polynomial as Pn


def radau_iia_tableau(s=3):
    """(a, b, c) of the s-stage Radau IIA method from the collocation
    definition."""
    p = Pn.polymul(Pn.polypow([0.0, 1.0], s - 1), Pn.polypow([-1.0, 1.0], s))
    dp = Pn.polyder(p, s - 1)
    c = np.sort(np.real(Pn.polyroots(dp)))
    c[-1] = 1.0
    a = np.zeros((s, s))
    for j in range(s):
        lj = np.array([1.0])
        for k in range(s):
            if k != j:
                lj = Pn.polymul(lj, np.array([-c[k], 1.0]) / (c[j] - c[k]))
        Ij = Pn.polyint(lj)
        for i in range(s):
            a[i, j] = Pn.polyval(c[i], Ij)
    return a, a[-1].copy(), c


class RadauIIA:
    def __init__(self, A_of_t, s=3, rtol=1e-12, atol=1e-16, h0=1e-9, h_max=np.inf,
                 max_steps=10_000_000):
        self.A_of_t = A_of_t
        self.a, self.b, self.c = radau_iia_tableau(s)
        self.s = s
        self.rtol, self.atol = rtol, atol
        self.h = h0
        self.h_max = h_max
        self.max_steps = max_steps
        self.n_steps = 0
        self.n_rejected = 0

    def step(self, t, y, h):
        """One collocation step of size h from (t, y)."""
        N, s = y.size, self.s
        M = np.eye(s * N)
        As = [self.A_of_t(t + self.c[j] * h) for j in range(s)]
        for i in range(s):
            for j in range(s):
                M[i * N:(i + 1) * N, j * N:(j + 1) * N] -= h * self.a[i, j] * As[j]
        Y = np.linalg.solve(M, np.tile(y, s))
        return Y[(s - 1) * N:]

    def integrate(self, t0, y0, t_out):
        """States at the sorted times t_out (t_out[0] may equal t0)."""
        t, y = float(t0), np.array(y0, dtype=np.float64)
        out = np.empty((len(t_out), y.size))
        order_exp = 1.0 / (self.s + 2)
        for k, tk in enumerate(t_out):
            while t < tk:
                if self.n_steps + self.n_rejected > self.max_steps:
                    raise RuntimeError("Radau IIA: step limit reached")
                h = min(self.h, self.h_max)
                last = t + h >= tk * (1.0 - 1e-15)
                if last:
                    h = tk - t
                y1 = self.step(t, y, h)
                yh = self.step(t, y, 0.5 * h)
                y2 = self.step(t + 0.5 * h, yh, 0.5 * h)
                sc = self.atol + self.rtol * max(np.abs(y).max(), np.abs(y2).max())
                err = np.abs(y2 - y1).max() / sc
                fac = 0.9 * (max(err, 1e-10)) ** (-order_exp)
                if err <= 1.0:
                    t = tk if last else t + h
                    y = y2
                    self.n_steps += 1
                    if not last:
                        self.h = h * min(4.0, fac)
                    elif fac < 1.0:
                        self.h = min(self.h, h * fac)
                else:
                    self.n_rejected += 1
                    self.h = h * max(0.1, fac)
            out[k] = y
        return out
