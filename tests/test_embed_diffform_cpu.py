"""The float32 difference form of D on a line object, emulated on the CPU.

The embedded float32 sweep evaluates e = D v on a line object (nodes
x_0 = a, x_1..x_m, x_N = b, end cells of length g_a, g_b, the rest h) as
    T_k - g_{k+1} T_{k+1} = q_k          (anti-causal, T_N = 0)
    e_k = g_k e_{k-1} + (1 - g_k^2) T_k  (causal, e_0 = 0)
plus A' e^{-alpha (x - a)} + B' e^{-alpha (b - x)} restoring e_N = 0, with q a
combination of second divided differences of v (uniform rows g_e, g_c, g_e;
two per-line coefficients on rows 1 and m).  This test derives those
coefficients here, in float64, from the quadrature's cell weights (the
exponential moments of the quadratic through three nodes), runs the two
recurrences with the kernel's work split (128 threads per line in 4 warps,
each thread a chunk of ceil((N + 1) / 128) nodes; chunk maps scanned over
the lanes of a warp, the warps' totals composed, each chunk re-run from its
carry) and compares with the oracle's v - L^{-1} v on line objects.
"""
import math

import numpy as np
import pytest

import oracle

THREADS = 128


def exp_moment(k, nu):
    """int_0^nu t^k e^{-t} dt (power series below 1, closed forms above)."""
    if nu < 1.0:
        term, s = nu ** (k + 1), 0.0
        for i in range(80):
            t = term / (k + 1 + i)
            s += t
            if abs(t) < 1e-18 * abs(s):
                break
            term *= -nu / (i + 1)
        return s
    e = math.exp(-nu)
    return [-math.expm1(-nu), 1 - (1 + nu) * e, 2 - (2 + nu * (2 + nu)) * e][k]


def cell_weights(s, length, a):
    """Weights on three nodes at signed distances s (from the cell's far end)
    of the quadratic interpolant integrated against alpha e^{-alpha y} over a
    cell of the given length."""
    nu = a * length
    M = [exp_moment(k, nu) for k in range(3)]
    w = []
    for i in range(3):
        sa, sb = s[(i + 1) % 3], s[(i + 2) % 3]
        w.append((M[2] - a * (sa + sb) * M[1] + a * a * sa * sb * M[0]) / (2 * a * a * (s[i] - sa) * (s[i] - sb)))
    return w


def positions(m, h, ga, gb):
    x = [0.0] + [ga + (j - 1) * h for j in range(1, m + 1)]
    return x + [x[m] + gb]


def beta_row(x, k, a):
    """Row k of the operator v -> q (the anti-causal right-hand side) as
    weights on the nodes 0..N."""
    N = len(x) - 1
    b = np.zeros(N + 1)
    g = lambda j: math.exp(-a * (x[j] - x[j - 1]))

    def add_left(j, c):          # J^L_j: the quadratic through x_{j-1}, x_j, x_{j+1} (x_{j-2} at the end)
        c0 = j - 1 if j + 1 <= N else j - 2
        w = cell_weights([x[j] - x[c0 + i] for i in range(3)], x[j] - x[j - 1], a)
        for i in range(3):
            b[c0 + i] += c * w[i]

    def add_right(j, c):         # J^R_j: the mirror rule on [x_j, x_{j+1}]
        c0 = j - 1 if j - 1 >= 0 else j
        w = cell_weights([x[c0 + i] - x[j] for i in range(3)], x[j + 1] - x[j], a)
        for i in range(3):
            b[c0 + i] += c * w[i]

    gk, gk1 = g(k), g(k + 1)
    ik, ik1 = 1 / (1 - gk * gk), 1 / (1 - gk1 * gk1)
    b[k] += ik + gk1 * gk1 * ik1
    b[k - 1] -= gk * ik
    b[k + 1] -= gk1 * ik1
    add_left(k, -ik)
    add_right(k - 1, gk * ik)
    add_left(k + 1, gk1 * ik1)
    add_right(k, -gk1 * gk1 * ik1)
    add_right(k, -1.0)
    return b


def dd_weight(x, t, j):
    """Weight of node j in the second divided difference at x_{t-1}, x_t, x_{t+1}."""
    p, c, n = x[t - 1], x[t], x[t + 1]
    if j == t - 1:
        return 2 / ((p - c) * (p - n))
    if j == t:
        return 2 / ((c - p) * (c - n))
    return 2 / ((n - p) * (n - c))


def line_constants(m, h, ga, gb, a):
    x = positions(m, h, ga, gb)
    N, h2 = m + 1, h * h
    L = dict(m=m, dA=math.exp(-a * ga), dB=math.exp(-a * gb), cA=-math.expm1(-2 * a * ga),
             cB=-math.expm1(-2 * a * gb), mu=math.exp(-a * x[N]), inv=1 / (-math.expm1(-2 * a * x[N])))
    L["rA"], L["rB"] = L["dA"] / math.exp(-a * h), L["dB"] / math.exp(-a * h)
    L["p1"] = 2 * h2 / ((x[2] - x[0]) * (x[2] - x[1]))
    L["q1"] = 2 * h2 / ((x[2] - x[0]) * (x[1] - x[0]))
    L["pm"] = 2 * h2 / ((x[N] - x[m - 1]) * (x[N] - x[m]))
    L["qm"] = 2 * h2 / ((x[N] - x[m - 1]) * (x[m] - x[m - 1]))
    b1 = beta_row(x, 1, a)
    L["g11"] = b1[0] / dd_weight(x, 1, 0) / h2
    L["g12"] = b1[3] / dd_weight(x, 2, 3) / h2 if m >= 2 else 0.0
    bm = beta_row(x, m, a)
    L["gNb"] = bm[N] / dd_weight(x, m, N) / h2
    L["gNa"] = bm[N - 3] / dd_weight(x, m - 1, N - 3) / h2 if m >= 2 else 0.0
    return L


def uniform_rows(h, a):
    """g_c, g_e of the interior rows: row 5 of a line of 9 interior nodes."""
    x = positions(9, h, h, h)
    b = beta_row(x, 5, a)
    ge = b[3] / dd_weight(x, 4, 3)
    gc = (b[4] - ge * dd_weight(x, 4, 4)) / dd_weight(x, 5, 4)
    return gc / (h * h), ge / (h * h)


def carries(p, q, forward):
    """The value entering each chunk, as the kernel forms it: the chunk maps
    y -> p y + q are scanned over the 32 lanes of each warp (inclusive,
    forward or from the right), the warps' totals are composed in order, and a
    lane's carry is its warp's incoming value pushed through the scanned maps
    of the lanes before it (forward) or after it (anti-causal)."""
    n = len(p)
    nw = n // 32
    P, Q = list(p), list(q)
    for w in range(nw):
        lanes = range(w * 32, w * 32 + 32) if forward else range(w * 32 + 31, w * 32 - 1, -1)
        accp, accq, first = 1.0, 0.0, True
        for i in lanes:
            if first:
                accp, accq, first = p[i], q[i], False
            else:
                accp, accq = p[i] * accp, p[i] * accq + q[i]
            P[i], Q[i] = accp, accq
    tot = [(P[w * 32 + 31], Q[w * 32 + 31]) if forward else (P[w * 32], Q[w * 32]) for w in range(nw)]
    out = []
    for i in range(n):
        w, lane = divmod(i, 32)
        yin = 0.0
        ws = range(0, w) if forward else range(nw - 1, w, -1)
        for u in ws:
            yin = tot[u][0] * yin + tot[u][1]
        if forward:
            out.append(yin if lane == 0 else P[i - 1] * yin + Q[i - 1])
        else:
            out.append(yin if lane == 31 else P[i + 1] * yin + Q[i + 1])
    return out


def diffform_D(v, L, h, a):
    m = L["m"]
    N = m + 1
    d, c = math.exp(-a * h), -math.expm1(-2 * a * h)
    gc, ge = uniform_rows(h, a)
    H = np.zeros(N + 1)
    H[1:m + 1] = v
    S = np.zeros(N + 1)
    for t in range(1, m + 1):
        if t == 1 or t == m:
            dn, dp = H[t + 1] - H[t], H[t] - H[t - 1]
            S[t] = L["p1"] * dn - L["q1"] * dp if t == 1 else L["pm"] * dn - L["qm"] * dp
        else:
            S[t] = (H[t + 1] - H[t]) - (H[t] - H[t - 1])
    Q = np.zeros(N + 1)
    for k in range(1, m + 1):
        if k == 1:
            Q[k] = L["g11"] * S[1] + (L["g12"] * S[2] if m >= 2 else 0.0)
        elif k == m:
            Q[k] = L["gNa"] * S[m - 1] + L["gNb"] * S[m]
        else:
            Q[k] = ge * (S[k - 1] + S[k + 1]) + gc * S[k]
    s = (N + THREADS) // THREADS
    chunks = [(min(t * s, N + 1), min(min(t * s, N + 1) + s, N + 1)) for t in range(THREADS)]
    # anti-causal: each thread reduces its chunk from the right, the chunk maps
    # compose right to left (lanes, then warps), each chunk re-runs from its carry
    p, q = [], []
    for k0, k1 in chunks:
        qq = 0.0
        for k in range(k1 - 1, k0 - 1, -1):
            g = L["dB"] if k == N - 1 else d
            qq = 0.0 if k == N else g * qq + Q[k]
        pp = d ** (k1 - k0) * (L["rB"] if k0 <= N - 1 < k1 else 1.0)
        p.append(pp)
        q.append(qq)
    cin = carries(p, q, forward=False)
    for t, (k0, k1) in enumerate(chunks):
        y = cin[t]
        for k in range(k1 - 1, k0 - 1, -1):
            g = L["dB"] if k == N - 1 else d
            y = 0.0 if k == N else g * y + Q[k]
            Q[k] = y
    # causal
    p, q = [], []
    for k0, k1 in chunks:
        qq = 0.0
        for k in range(k0, k1):
            g = L["dA"] if k == 1 else (L["dB"] if k == N else d)
            cg = L["cA"] if k == 1 else (L["cB"] if k == N else c)
            qq = 0.0 if k == 0 else g * qq + cg * Q[k]
        pp = d ** (k1 - k0) * (L["rA"] if k0 <= 1 < k1 else 1.0) * (L["rB"] if k0 <= N < k1 else 1.0)
        p.append(pp)
        q.append(qq)
    cin = carries(p, q, forward=True)
    for t, (k0, k1) in enumerate(chunks):
        y = cin[t]
        for k in range(k0, k1):
            g = L["dA"] if k == 1 else (L["dB"] if k == N else d)
            cg = L["cA"] if k == 1 else (L["cB"] if k == N else c)
            y = 0.0 if k == 0 else g * y + cg * Q[k]
            Q[k] = y
    Bp = -Q[N] * L["inv"]
    Ap = -Bp * L["mu"]
    return np.array([Q[k] + Ap * L["dA"] * d ** (k - 1) + Bp * L["dB"] * d ** (m - k) for k in range(1, m + 1)])


@pytest.mark.parametrize("m", [1, 2, 3, 5, 130, 903])
@pytest.mark.parametrize("gaps", [(1.0, 1.0), (0.3, 0.9), (1e-4, 0.5), (0.99, 1e-6)])
@pytest.mark.parametrize("nu", [0.05, 0.9, 4.0])
def test_difference_form_matches_the_oracle(m, gaps, nu):
    """float64 throughout; the end triples' weights reach h / g = 1e6 at the
    smallest gap, so agreement is to about 1e6 rounding units (bound 1e-8)."""
    h = 0.01
    a = nu / h
    ga, gb = gaps[0] * h, gaps[1] * h
    v = np.random.default_rng(m + int(1e3 * nu)).normal(size=m)
    e = diffform_D(v, line_constants(m, h, ga, gb, a), h, a)
    ref = v - oracle.linv_obj(v, h, ga, gb, a)
    assert np.abs(e - ref).max() <= 1e-8 * np.abs(ref).max()
