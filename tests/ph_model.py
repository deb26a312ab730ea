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


def particular_skewed_df1(coef, xb, m_cap=None, dtype=np.float64):
    """The skewed-pass kernel's particular solution of every lane block (rows of xb), in the
    kernel's direct-form-I order: section k runs its poles on F_k (its input already through its
    own numerator), y = F_k - a1 y[-1] - a2 y[-2], and then applies section k+1's numerator to its
    output history, F_{k+1} = b0' y + b1' y[-1] + b2' y[-2]; section 0's F is the numerator on the
    input.  Sections run skewed, section k taking sample i - k at step i with the F that section
    k-1 formed at step i-1, every step visiting the sections from the last down.  Returns the
    outputs, the terminal transposed-direct-form-II states formed from each section's last two
    inputs and outputs, and (with m_cap) the state after sample m_cap.

    With dtype=np.float32 every multiply-add is rounded to float32 once (a fused multiply-add: the
    float32 product is exact in float64), as on the GPU."""
    K = len(coef)
    nl, N = xb.shape
    f = dtype

    def fma(a, b, c):
        return (np.float64(a) * np.asarray(b, np.float64) + np.asarray(c, np.float64)).astype(f)

    x = xb.astype(f)
    y1 = np.zeros((K, nl), f)
    y2 = np.zeros((K, nl), f)
    pipe = np.zeros((K, nl), f)
    x1 = np.zeros(nl, f)
    x2 = np.zeros(nl, f)
    cap = np.zeros((K, 2, nl), f)
    out = np.zeros((nl, N), f)
    cf = [tuple(f(v) for v in c) for c in coef]
    for i in range(N + K - 1):
        for k in range(K - 1, -1, -1):
            m = i - k
            if m < 0 or m >= N:
                continue
            b0, b1, b2, a1, a2 = cf[k]
            if k == 0:
                xin1, xin2 = x[:, i], x1
                F = fma(b1, x1, fma(b2, x2, (np.float64(b0) * x[:, i]).astype(f)))
            else:
                xin1, xin2 = y1[k - 1], y2[k - 1]
                F = pipe[k - 1]
            y = fma(-a1, y1[k], fma(-a2, y2[k], F))
            if m_cap is not None and m == m_cap:
                cap[k, 0] = fma(b1, xin1, fma(b2, xin2, fma(-a1, y, (np.float64(-a2) * y1[k]).astype(f))))
                cap[k, 1] = fma(b2, xin1, (np.float64(-a2) * y).astype(f))
            if k + 1 < K:
                n0, n1, n2 = cf[k + 1][:3]
                pipe[k] = fma(n1, y1[k], fma(n2, y2[k], (np.float64(n0) * y).astype(f)))
            else:
                out[:, m] = y
            y2[k], y1[k] = y1[k], y
            if k == 0:
                x2, x1 = x1, x[:, i]
    z = np.zeros((nl, 2 * K), f)
    for k, (b0, b1, b2, a1, a2) in enumerate(cf):
        xi1, xi2 = (x1, x2) if k == 0 else (y1[k - 1], y2[k - 1])
        z[:, 2 * k] = fma(b1, xi1, fma(b2, xi2, fma(-a1, y1[k], (np.float64(-a2) * y2[k]).astype(f))))
        z[:, 2 * k + 1] = fma(b2, xi1, (np.float64(-a2) * y1[k]).astype(f))
    capz = None
    if m_cap is not None:
        capz = np.zeros((nl, 2 * K), f)
        capz[:, 0::2] = cap[:, 0].T
        capz[:, 1::2] = cap[:, 1].T
    return out, z, capz
