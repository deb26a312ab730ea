"""Float64 step-by-step model of the GPU kernel's algorithm (a test aid, not the oracle).

It follows the same steps, in the same order and with the same tables, as the
sm_103a kernel, so that the algebra can be checked on the CPU against the
oracle (which is the plain recurrence) and against dense solves.

Notation (per section; ``a1, a2`` feedback, ``b0, b1, b2`` feed-forward):

* a group of ``C = N*L`` samples; lane ``l`` owns the contiguous samples
  ``l*N + m``, ``m = 0..N-1`` (Sec. IV-A); block ``m`` of the stride-N
  permuted system of Eq. 2-3 is register ``m`` across the lanes;
* reduction levels (Sec. II-E, Eqs. 14-23): ``e_0 = a1, f_0 = a2``,
  ``e_{i+1} = 2 f_i - e_i^2, f_{i+1} = f_i^2``; level ``i`` holds the
  recurrence ``y[m] + e_i y[m - 2^i] + f_i y[m - 2^{i+1}] = v_i[m]``;
* the divide-and-conquer first level multiplies both sides by ``A(-z)``, so
  ``v_1 = B(z) A(-z) x`` (the five taps ``1, d_B, e_B, c_B, f_B`` of Eq. 23
  when ``b0 = 1``) on every sample; the odd chain keeps ``m = -1 mod 2^i`` and
  the even chain ``m = -2 mod 2^i``; after ``D = log2 N`` levels the lane's
  two terminal samples ``N-1`` and ``N-2`` are exposed at once;
* each lane is solved under zero incoming state; the lane's terminal state in
  transposed direct form II is scanned across lanes with the N-step
  transition ``T^N`` (``T = [[-a1, 1], [-a2, 0]]``), and across groups with
  ``T^C`` (Eq. 25, by decoupled lookback on the GPU);
* once a lane's incoming state ``z`` is known, it enters the lane's system as
  ``z1`` at sample 0 and ``z2`` at sample 1 of the right-hand side; after the
  reduction this is ``Q_i[m] z1 + Q_i[m-1] z2`` with
  ``Q_i(z) = prod_{j<i} A_j(-z^{2^j})``, non-zero only for ``m < 2^{i+1}``;
  back substitution then recovers every sample with the state included (the
  homogeneous correction of Eq. 24 folded into it).
"""
from __future__ import annotations

import numpy as np


def poly_mul(p, q):
    return np.convolve(np.asarray(p, dtype=np.float64), np.asarray(q, dtype=np.float64))


def level_coeffs(a1, a2, D):
    e, f = [a1], [a2]
    for i in range(D):
        e.append(2 * f[i] - e[i] ** 2)
        f.append(f[i] ** 2)
    return e, f


def q_tables(a1, a2, D):
    """Q_i for i = 0..D as coefficient arrays in z^-1."""
    e, f = level_coeffs(a1, a2, D)
    Q = [np.array([1.0])]
    for i in range(D):
        s = 1 << i
        g = np.zeros(2 * s + 1)
        g[0], g[s], g[2 * s] = 1.0, -e[i], f[i]
        Q.append(poly_mul(Q[i], g))
    return Q


def first_level_taps(b0, b1, b2, a1, a2):
    """B(z) A(-z): five taps on x for the divide-and-conquer first level (Eq. 23 when b0 = 1)."""
    return poly_mul([b0, b1, b2], [1.0, -a1, a2])


def transition(a1, a2):
    return np.array([[-a1, 1.0], [-a2, 0.0]])


def chain_points(N, i, parity):
    """S_i of the odd (parity 1) or even (parity 0) chain inside a lane."""
    s = 1 << i
    off = s - 1 if parity else s - 2
    return list(range(off, N, s))


def lane_reduce(x, taps, e, f, N, D):
    """Zero-state reduction of one lane. Returns the v_i arrays (NaN where not formed)."""
    v = {1: np.array([sum(taps[k] * (x[m - k] if m - k >= 0 else 0.0) for k in range(5)) for m in range(N)])}
    for i in range(1, D):
        s = 1 << i
        nxt = np.full(N, np.nan)
        for par in (0, 1):
            for m in chain_points(N, i + 1, par):
                a = v[i][m]
                b = v[i][m - s] if m - s >= 0 else 0.0
                c = v[i][m - 2 * s] if m - 2 * s >= 0 else 0.0
                nxt[m] = a - e[i] * b + f[i] * c
        v[i + 1] = nxt
    return v


def lane_terminal_state(x, v, D, N, b1, b2, a1, a2):
    yo, ye = v[D][N - 1], v[D][N - 2]
    return np.array([b1 * x[N - 1] + b2 * x[N - 2] - a1 * yo - a2 * ye, b2 * x[N - 1] - a2 * yo])


def lane_back_substitute(v, Q, e, f, N, D, z):
    y = np.full(N, np.nan)

    def inj(i, m):
        q = Q[i]
        t = q[m] * z[0] if m < len(q) else 0.0
        if 0 <= m - 1 < len(q):
            t += q[m - 1] * z[1]
        return t

    y[N - 1] = v[D][N - 1] + inj(D, N - 1)
    y[N - 2] = v[D][N - 2] + inj(D, N - 2)
    for i in range(D - 1, 0, -1):
        s = 1 << i
        for par in (1, 0):
            keep = set(chain_points(N, i + 1, par))
            for m in chain_points(N, i, par):
                if m in keep:
                    continue
                val = v[i][m] + inj(i, m)
                if m - s >= 0:
                    val -= e[i] * y[m - s]
                if m - 2 * s >= 0:
                    val -= f[i] * y[m - 2 * s]
                y[m] = val
    # level-1 chains cover every sample; in the kernel the N = 2 case stops at D = 1
    return y


def filter_section_group_lanes(x, coef, N, L, z_in_group, taps=None):
    """One section over one group: returns (y, t_group_zero_state, lane incoming states)."""
    b0, b1, b2, a1, a2 = coef
    D = int(round(np.log2(N)))
    e, f = level_coeffs(a1, a2, D)
    Q = q_tables(a1, a2, D)
    taps = first_level_taps(b0, b1, b2, a1, a2) if taps is None else taps
    TN = np.linalg.matrix_power(transition(a1, a2), N)
    lanes = x.reshape(L, N)
    vs, ts = [], []
    for l in range(L):
        v = lane_reduce(lanes[l], taps, e, f, N, D)
        vs.append(v)
        ts.append(lane_terminal_state(lanes[l], v, D, N, b1, b2, a1, a2))
    # lane scan under zero group state (inclusive)
    Z = []
    acc = np.zeros(2)
    for l in range(L):
        acc = ts[l] + TN @ acc
        Z.append(acc.copy())
    t_group = Z[-1]
    y = np.empty(N * L)
    zins = []
    for l in range(L):
        zin = (Z[l - 1] if l else np.zeros(2)) + np.linalg.matrix_power(TN, l) @ z_in_group
        zins.append(zin)
        y[l * N:(l + 1) * N] = lane_back_substitute(vs[l], Q, e, f, N, D, zin)
    return y, t_group, zins


def lookback_compose(t_locals, glob, TC, window=32):
    """Incoming state of group g from predecessors g-1, g-2, ...: locals until the first global.

    ``t_locals[k]`` is the zero-state carry of group g-1-k (k < j), ``glob`` the
    resolved carry of group g-1-j.  Composes in windows of ``window`` like the
    warp-parallel lookback: sum_k TC^k t_k + TC^j glob.
    """
    j = len(t_locals)
    acc = np.zeros(2)
    mult = np.eye(2)
    for w0 in range(0, j + 1, window):
        part = np.zeros(2)
        for k in range(w0, min(j + 1, w0 + window)):
            val = t_locals[k] if k < j else glob
            part += np.linalg.matrix_power(TC, k - w0) @ val
        acc += mult @ part
        mult = mult @ np.linalg.matrix_power(TC, window)
    return acc


def sosfilt_model(sos, x, N, L, zi=None, normalize=False):
    """Whole cascade over a signal, group by group; returns (y, zf)."""
    sos = np.asarray(sos, dtype=np.float64).reshape(-1, 5)
    K = sos.shape[0]
    x = np.asarray(x, dtype=np.float64)
    n = x.shape[0]
    C = N * L
    G = max(1, -(-n // C))
    zi = np.zeros((K, 2)) if zi is None else np.asarray(zi, dtype=np.float64).reshape(K, 2)
    coefs = sos.copy()
    scale_in = 1.0
    zscale = np.ones(K)
    if normalize:
        b0 = sos[:, 0]
        coefs[:, :3] = sos[:, :3] / b0[:, None]
        scale_in = float(np.prod(b0))
        # section k's output and state are carried as prod_{j>k} b0_j times their true values
        zscale = np.array([np.prod(b0[k + 1:]) for k in range(K)])
    xp = np.zeros(G * C)
    xp[:n] = x * scale_in
    carries = [zi[k] * zscale[k] for k in range(K)]  # incoming state of the current group per section
    zf = np.zeros((K, 2))
    out = np.empty(G * C)
    for g in range(G):
        cur = xp[g * C:(g + 1) * C]
        for k in range(K):
            b0, b1, b2, a1, a2 = coefs[k]
            TN = np.linalg.matrix_power(transition(a1, a2), N)
            TC = np.linalg.matrix_power(TN, L)
            ycur, t_group, _ = filter_section_group_lanes(cur, coefs[k], N, L, carries[k])
            if g == G - 1:
                p = n - 1 - g * C  # last real sample of the signal in this group
                if n == 0:
                    zf[k] = zi[k] * zscale[k]
                else:
                    xm1 = cur[p - 1] if p >= 1 else None
                    ym1 = ycur[p - 1] if p >= 1 else None
                    if p == 0:  # previous sample lies in the previous group: use the carried state
                        zprev = carries[k]
                        z1 = b1 * cur[0] - a1 * ycur[0] + zprev[1]
                        z2 = b2 * cur[0] - a2 * ycur[0]
                    else:
                        z1 = b1 * cur[p] + b2 * xm1 - a1 * ycur[p] - a2 * ym1
                        z2 = b2 * cur[p] - a2 * ycur[p]
                    zf[k] = [z1, z2]
            carries[k] = t_group + TC @ carries[k]
            cur = ycur
        out[g * C:(g + 1) * C] = cur
    zf = zf / zscale[:, None]
    return out[:n], zf
