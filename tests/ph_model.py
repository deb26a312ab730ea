"""Float64 step model of the PH-factorization kernel's algorithm (a test aid, not the oracle).

It follows the kernel's decomposition, in the kernel's order and with the kernel's tables, so that
the algebra can be checked on the CPU against the oracle (the plain recurrence):

* lane ``l`` of a group of ``C = N*L`` samples owns samples ``l*N .. l*N+N-1`` (Sec. IV-A);
* particular solutions (Sec. II-C, forward substitution from zero initial blocks): for every
  section in turn, each lane runs the section's recurrence over its ``N`` samples from zero
  state; the input of section ``k`` is the particular output of section ``k-1``;
* the cascade state is ``2K`` words (transposed direct form II, ``(z1, z2)`` per section); ``M1``
  is its one-sample zero-input transition and ``M_N = M1^N``, block lower-triangular;
* lane scan: with ``t_l`` the lane's terminal particular state, the lane's incoming state relative
  to zero group state is ``S_0 = 0, S_{l+1} = M_N S_l + t_l``, computed section by section:
  ``u_l = t_l[k] + sum_{j<k} M_N[k][j] S_l[j]`` then ``E_l = T_k^N E_{l-1} + u_l`` and
  ``S_l[k] = E_{l-1}``; ``E_{L-1}`` is the group's local carry;
* groups of a tile and tiles: ``Z_{v+1} = A_C Z_v + a_v`` with ``A_C = M_N^L``, tiles of ``W``
  groups with ``A_T = A_C^W`` (Eq. 25 on the cascade state);
* correction (Eq. 24 in cascade form): ``y[lN + m] = w[lN + m] + sum_j H_j(m) (S_l + M_N^l Z)_j``
  with ``H_j(m)`` the cascade's zero-input output at ``m`` from unit state ``j``;
* final state: the lane-local particular state after the last sample plus ``M1^(m+1)`` applied to
  the lane's true incoming state.
"""
from __future__ import annotations

import numpy as np


def _step(coef, z, x):
    """One sample through the cascade (TDF-II), z updated in place; returns the output."""
    v = x
    for k, (b0, b1, b2, a1, a2) in enumerate(coef):
        y = b0 * v + z[2 * k]
        z[2 * k] = b1 * v - a1 * y + z[2 * k + 1]
        z[2 * k + 1] = b2 * v - a2 * y
        v = y
    return v


def tables(coef, N):
    K = len(coef)
    S = 2 * K
    M1 = np.zeros((S, S))
    H = np.zeros((S, N))
    for j in range(S):
        z = np.zeros(S)
        z[j] = 1.0
        _step(coef, z, 0.0)
        M1[:, j] = z
        h = np.zeros(S)
        h[j] = 1.0
        for m in range(N):
            H[j, m] = _step(coef, h, 0.0)
    return M1, H


def particular(coef, xb):
    """Particular solutions of every lane block (rows of xb) through the whole cascade, with the
    lane-local states after each sample (for the final state)."""
    K = len(coef)
    nl, N = xb.shape
    w = xb.astype(np.float64).copy()
    states = np.zeros((nl, N, 2 * K))
    for k, (b0, b1, b2, a1, a2) in enumerate(coef):
        x = w.copy()
        x1 = np.zeros(nl)
        x2 = np.zeros(nl)
        w1 = np.zeros(nl)
        w2 = np.zeros(nl)
        for m in range(N):
            xm = x[:, m]
            wm = b0 * xm + b1 * x1 + b2 * x2 - a1 * w1 - a2 * w2
            w[:, m] = wm
            states[:, m, 2 * k] = b1 * xm + b2 * x1 - a1 * wm - a2 * w1
            states[:, m, 2 * k + 1] = b2 * xm - a2 * wm
            x2, x1, w2, w1 = x1, xm, w1, wm
    return w, states


def ph_filter(sos, x, zi=None, N=32, L=32, W=8, anchored=False):
    """Filter x as the kernel does; returns (y, zf).  With anchored, a tile's incoming state is
    composed as the PH kernels' lookback does it: the resolved carry of the anchor tile (the last
    multiple of 32 before it) and the local carries of the tiles after the anchor, each carried
    forward with its power of A_T; only anchors resolve (inclusive = A_T Z + local carry)."""
    coef = [tuple(float(v) for v in row) for row in np.asarray(sos, dtype=np.float64).reshape(-1, 5)]
    K = len(coef)
    S = 2 * K
    n = len(x)
    C = N * L
    G = max(1, -(-n // C))
    xp = np.zeros(G * C)
    xp[:n] = np.asarray(x, dtype=np.float64)
    M1, H = tables(coef, N)
    MN = np.linalg.matrix_power(M1, N)
    AC = np.linalg.matrix_power(MN, L)
    AT = np.linalg.matrix_power(AC, W)
    w, states = particular(coef, xp.reshape(G * L, N))
    # terminal particular state of every lane
    t = states[:, N - 1, :].reshape(G, L, S)
    # lane scan, section by section, relative to zero group state
    Sl = np.zeros((G, L, S))
    a = np.zeros((G, S))
    for k in range(K):
        u = t[:, :, 2 * k:2 * k + 2].copy()
        for j in range(k):
            u += Sl[:, :, 2 * j:2 * j + 2] @ MN[2 * k:2 * k + 2, 2 * j:2 * j + 2].T
        Tk = MN[2 * k:2 * k + 2, 2 * k:2 * k + 2]
        E = np.zeros((G, 2))
        for l in range(L):
            Sl[:, l, 2 * k:2 * k + 2] = E
            E = E @ Tk.T + u[:, l]
        a[:, 2 * k:2 * k + 2] = E
    # tiles of W groups, then the groups of each tile
    n_tiles = -(-G // W)
    Zg = np.zeros((G, S))
    z0 = np.zeros(S) if zi is None else np.asarray(zi, dtype=np.float64).reshape(S).copy()
    local = np.zeros((n_tiles, S))  # tile carries under zero incoming state (the fold)
    for tt in range(n_tiles):
        c = None
        for v in range(W):
            g = tt * W + v
            ag = a[g] if g < G else np.zeros(S)
            c = ag.copy() if c is None else AC @ c + ag
        local[tt] = c
    Ztile = np.zeros((n_tiles, S))
    if anchored:
        resolved = {}
        ATp = [np.linalg.matrix_power(AT, d) for d in range(33)]
        for tt in range(n_tiles):
            if tt == 0:
                Ztile[tt] = z0
            else:
                anchor = ((tt - 1) // 32) * 32
                z = ATp[tt - 1 - anchor] @ resolved[anchor]
                for pred in range(anchor + 1, tt):
                    z = z + ATp[tt - 1 - pred] @ local[pred]
                Ztile[tt] = z
            if tt % 32 == 0:
                resolved[tt] = AT @ Ztile[tt] + local[tt]
    else:
        Zt = z0
        for tt in range(n_tiles):
            Ztile[tt] = Zt
            Zt = AT @ Zt + local[tt]
    for tt in range(n_tiles):
        z = Ztile[tt].copy()
        for v in range(W):
            g = tt * W + v
            if g < G:
                Zg[g] = z
                z = AC @ z + a[g]
    # correction, one pass over the samples
    Ml = [np.linalg.matrix_power(MN, l) for l in range(L)]
    y = w.reshape(G, L, N).copy()
    true_state = np.zeros((G, L, S))
    for l in range(L):
        true_state[:, l] = Sl[:, l] + Zg @ Ml[l].T
        y[:, l, :] += true_state[:, l] @ H
    y = y.reshape(-1)[:n]
    # final state after the last sample
    p_last = n - 1 - (G - 1) * C
    l_last, m_last = divmod(p_last, N)
    zf = states[(G - 1) * L + l_last, m_last] + np.linalg.matrix_power(M1, m_last + 1) @ true_state[G - 1, l_last]
    return y, zf


def particular_skewed_df2(coef, xb, m_cap=None):
    """The skewed-pass kernel's particular solution of every lane block (rows of xb): direct form II
    sections (u = x - a1 u[-1] - a2 u[-2], w = b0 u + b1 u[-1] + b2 u[-2]) run skewed, section k
    taking sample i - k at step i with section k-1's output of step i-1 as input, every step visiting
    the sections from the last down.  Returns the outputs, the terminal transposed-direct-form-II
    states converted from the last two u of each section, and (with m_cap) the converted state after
    sample m_cap."""
    K = len(coef)
    nl, N = xb.shape
    x = xb.astype(np.float64)
    u1 = np.zeros((K, nl))
    u2 = np.zeros((K, nl))
    pipe = np.zeros((K, nl))
    cap = np.zeros((K, 2, nl))
    out = np.zeros((nl, N))
    for i in range(N + K - 1):
        for k in range(K - 1, -1, -1):
            m = i - k
            if m < 0 or m >= N:
                continue
            b0, b1, b2, a1, a2 = coef[k]
            xin = x[:, i] if k == 0 else pipe[k - 1]
            u = xin - a2 * u2[k] - a1 * u1[k]
            w = b0 * u + b1 * u1[k] + b2 * u2[k]
            u2[k], u1[k] = u1[k], u
            if k == K - 1:
                out[:, m] = w
            else:
                pipe[k] = w
            if m_cap is not None and m == m_cap:
                cap[k, 0], cap[k, 1] = u1[k], u2[k]

    def convert(ua, ub):
        z = np.zeros((nl, 2 * K))
        for k, (b0, b1, b2, a1, a2) in enumerate(coef):
            z[:, 2 * k] = (b1 - b0 * a1) * ua[k] + (b2 - b0 * a2) * ub[k]
            z[:, 2 * k + 1] = (b2 - b0 * a2) * ua[k] + (a1 * b2 - a2 * b1) * ub[k]
        return z

    return out, convert(u1, u2), (convert(cap[:, 0], cap[:, 1]) if m_cap is not None else None)
