"""Generate alpert_rules.h: one-sided endpoint corrections of the hybrid
Gauss-trapezoidal rule (Sec. 3.4), used by the library's contour quadrature.

The paper prints only kappa = 7 for p = 8; the nodes/weights are derived from
the defining conditions.  The corrected rule
    h sum_k w_k f(a + x_k h) + h sum_{j>=0} f(a + (kappa + j) h)
is exact to O(h^{2p}) iff  sum_k w_k x_k^m = B_{m+1}(kappa)/(m+1), m < 2p
(Euler-Maclaurin with Hurwitz-zeta regularisation).  Here the moments are
computed with B_{m+1}(kappa)/(m+1) = B_{m+1}/(m+1) + sum_{j=0}^{kappa-1} j^m,
turned into three-term recurrence coefficients by Chebyshev's algorithm, and
the nodes/weights taken as eigenvalues / squared first eigenvector components
of the Jacobi matrix (Golub-Welsch), all in 80-digit arithmetic (mpmath).

    python paper_2001_06113_gb300/csrc/gen_alpert.py > paper_2001_06113_gb300/csrc/alpert_rules.h
"""
from __future__ import annotations

import mpmath as mp

RULES = [(4, 4), (8, 7)]   # (p, kappa)


def moments(p: int, kappa: int):
    out = []
    for m in range(2 * p):
        s = mp.bernoulli(m + 1) / (m + 1)
        s += sum(mp.mpf(j) ** m if not (j == 0 and m == 0) else mp.mpf(1) for j in range(kappa))
        out.append(s)
    return out


def chebyshev_algorithm(mom, n):
    """Recurrence coefficients alpha_k, beta_k (k < n) from 2n moments."""
    sig_prev = [mp.mpf(0)] * (2 * n)
    sig = list(mom)
    alpha = [mom[1] / mom[0]]
    beta = [mom[0]]
    for k in range(1, n):
        new = [mp.mpf(0)] * (2 * n)
        for l in range(k, 2 * n - k):
            new[l] = sig[l + 1] - alpha[k - 1] * sig[l] - beta[k - 1] * sig_prev[l]
        alpha.append(new[k + 1] / new[k] - sig[k] / sig[k - 1])
        beta.append(new[k] / sig[k - 1])
        sig_prev, sig = sig, new
    return alpha, beta


def rule(p, kappa):
    mp.mp.dps = 80
    a, b = chebyshev_algorithm(moments(p, kappa), p)
    J = mp.zeros(p, p)
    for i in range(p):
        J[i, i] = a[i]
        if i + 1 < p:
            J[i, i + 1] = J[i + 1, i] = mp.sqrt(b[i + 1])
    E, Q = mp.eigsy(J)
    pts = sorted((E[i], b[0] * Q[0, i] ** 2) for i in range(p))
    return [x for x, _ in pts], [w for _, w in pts]


def main():
    print("// Generated by gen_alpert.py (Chebyshev algorithm + Golub-Welsch, 80 digits).")
    print("// One-sided Alpert endpoint corrections: nodes x_k in (0, kappa), weights w_k.")
    print("#pragma once")
    print("namespace tdse {")
    print("struct AlpertRule { int p, kappa; const double* x; const double* w; };")
    for p, kappa in RULES:
        x, w = rule(p, kappa)
        print(f"static const double kAlpertX{p}[{p}] = {{" + ", ".join(mp.nstr(v, 20) for v in x) + "};")
        print(f"static const double kAlpertW{p}[{p}] = {{" + ", ".join(mp.nstr(v, 20) for v in w) + "};")
    print("static const AlpertRule kAlpertRules[] = {" +
          ", ".join(f"{{{p}, {k}, kAlpertX{p}, kAlpertW{p}}}" for p, k in RULES) + "};")
    print("}  // namespace tdse")


if __name__ == "__main__":
    main()
