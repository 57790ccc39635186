"""Exact generators and operator products on tiny lattices (test infrastructure).

Builds the Markov generator of Eq. generator as a sparse matrix over the whole
configuration space, straight from the paper's rate formulas, written per
site (Eq. adsdesrate, Eq. Arrhenius, Table COrates). It does not use the
oracle's class tables or member lists, so it can pin them.

Conventions: site i = y*lx + x on a periodic lattice, state code
sum_i sigma_i * base**i, neighbour directions N, E, S, W. A distribution is
a row vector p; it evolves as p e^{tQ}. Events are split into the E and O
parts of Eq. opdecomp by the ownership rule: a site event belongs to its
cell; a bond inside a cell to that cell; a horizontal bond crossing a cell
edge to the E colour, a vertical one to the O colour.
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp
from scipy.sparse.linalg import expm_multiply

DIRS = [(0, -1), (1, 0), (0, 1), (-1, 0)]


def _nb(lx, ly, i, d):
    x, y = i % lx, i // lx
    dx, dy = DIRS[d]
    return ((y + dy) % ly) * lx + (x + dx) % lx


def decode(lx, ly, base):
    """All configurations: array (base**N, N) of site values."""
    N = lx * ly
    codes = np.arange(base ** N, dtype=np.int64)
    out = np.empty((codes.size, N), np.int8)
    for i in range(N):
        out[:, i] = (codes // base ** i) % base
    return out


def events(lx, ly, model, rates, S=None):
    """Every transition of the model on every configuration (or on the rows of S).

    Yields (owner, sites, new_values, rate_vector) where owner describes the
    event for the E/O split: ('site', i) or ('bond', i, d).
    The rate formulas are the paper's, per site:
      ADSDES     c(x) = ka (1 - s_x) + kd s_x exp(-beta U), U = J sum_nn s_y
      ISING      c(x) = ka (1 - s_x) + kd s_x exp(-beta U), U = K sum_nn s_y - h,
                 K = 4J, h = 2K (zero spin field)
      ISING1D    the same on a ring (ly = 1, neighbours x-1 and x+1 only),
                 beta K = betaJ and beta h = betah given freely (Section 7)
      DIFFUSION  ADSDES flips, plus a hop x->y (|x-y| = 1) of a particle at x to
                 an empty y with rate nu exp(-beta J sum_{z nn x} s_z)
      ZGB        Table COrates with A = the single-site adsorber, B = the
                 dissociative adsorber: A adsorbs on an empty site at yA;
                 B2 adsorbs at an empty x with rate (1-yA) nu_0(x)/4 onto x and a
                 uniformly chosen empty neighbour; A at x reacts with rate
                 kr nu_B(x)/4 with a uniformly chosen B neighbour (and B at x
                 with rate kr nu_A(x)/4 with an A neighbour), both sites empty
                 after; A desorbs at kd.
    """
    N = lx * ly
    base = 3 if model == "ZGB" else 2
    if S is None:
        S = decode(lx, ly, base)
    ka, kd, bJ = rates.get("ka", 1.0), rates.get("kd", 1.0), rates.get("betaJ", 0.0)
    dirs = (1, 3) if model == "ISING1D" else range(4)
    nn_occ = np.stack([sum((S[:, _nb(lx, ly, i, d)] == 1).astype(np.int64) for d in dirs)
                       for i in range(N)], axis=1)
    out = []
    if model in ("ADSDES", "ISING", "DIFFUSION", "ISING1D"):
        for i in range(N):
            s = S[:, i].astype(np.float64)
            if model == "ISING":
                K, h = 4.0 * bJ, 8.0 * bJ  # beta*K and beta*h
                U = K * nn_occ[:, i] - h
            elif model == "ISING1D":
                U = bJ * nn_occ[:, i] - rates.get("betah", 0.0)
            else:
                U = bJ * nn_occ[:, i]
            c = ka * (1 - s) + kd * s * np.exp(-U)
            out.append((("site", i), (i,), (1 - S[:, i],), c))
    if model == "DIFFUSION":
        nu = rates.get("nu", 0.0)
        for i in range(N):
            for d in range(4):
                j = _nb(lx, ly, i, d)
                ok = (S[:, i] == 1) & (S[:, j] == 0)
                c = np.where(ok, nu * np.exp(-bJ * nn_occ[:, i]), 0.0)
                out.append((("bond", i, d), (i, j), (np.zeros(len(S), np.int8),
                                                     np.ones(len(S), np.int8)), c))
    if model == "ZGB":
        yA, kr = rates.get("yA", 0.0), rates.get("kr", 0.0)
        zeros = np.zeros(len(S), np.int8)
        for i in range(N):
            empty = S[:, i] == 0
            out.append((("site", i), (i,), (np.ones(len(S), np.int8),), np.where(empty, yA, 0.0)))
            out.append((("site", i), (i,), (zeros,), np.where(S[:, i] == 1, kd, 0.0)))
            nu0 = sum((S[:, _nb(lx, ly, i, d)] == 0).astype(np.int64) for d in range(4))
            nuA = sum((S[:, _nb(lx, ly, i, d)] == 1).astype(np.int64) for d in range(4))
            nuB = sum((S[:, _nb(lx, ly, i, d)] == 2).astype(np.int64) for d in range(4))
            for d in range(4):
                j = _nb(lx, ly, i, d)
                # B2: total (1-yA) nu_0/4 at x, the partner uniform among the
                # nu_0 empty neighbours -> (1-yA)/4 per (x, empty y)
                tot = np.where(empty, (1 - yA) * nu0 / 4.0, 0.0)
                pick = np.where(S[:, j] == 0, 1.0 / np.maximum(nu0, 1), 0.0)
                out.append((("bond", i, d), (i, j), (2 * np.ones(len(S), np.int8),
                                                     2 * np.ones(len(S), np.int8)), tot * pick))
                # reaction seen from x: A with a B neighbour, or B with an A one
                totA = np.where(S[:, i] == 1, kr * nuB / 4.0, 0.0)
                pickA = np.where(S[:, j] == 2, 1.0 / np.maximum(nuB, 1), 0.0)
                totB = np.where(S[:, i] == 2, kr * nuA / 4.0, 0.0)
                pickB = np.where(S[:, j] == 1, 1.0 / np.maximum(nuA, 1), 0.0)
                out.append((("bond", i, d), (i, j), (zeros, zeros), totA * pickA + totB * pickB))
    return S, base, out


def owner_colour(lx, ly, qx, qy, owner):
    """Colour (0 = E, 1 = O) whose generator holds the event."""
    if owner[0] == "site":
        i = owner[1]
        cx, cy = (i % lx) // qx, (i // lx) // qy
        return (cx + cy) % 2
    _, i, d = owner
    x, y = i % lx, i // lx
    cx, cy = x // qx, y // qy
    dx, dy = DIRS[d]
    nx, ny = x + dx, y + dy
    inside = (0 <= nx - cx * qx < qx) and (0 <= ny - cy * qy < qy)
    if inside:
        return (cx + cy) % 2
    return 0 if dx != 0 else 1


def generator(lx, ly, model, rates, qx=None, qy=None, colour=None):
    """Sparse generator Q (rows = from). With colour given, only that part."""
    S, base, evs = events(lx, ly, model, rates)
    nstate = len(S)
    pw = base ** np.arange(lx * ly, dtype=np.int64)
    codes = S.astype(np.int64) @ pw
    rows, cols, vals = [], [], []
    for owner, sites, newv, c in evs:
        if colour is not None and owner_colour(lx, ly, qx, qy, owner) != colour:
            continue
        nz = c > 0
        if not nz.any():
            continue
        tgt = codes.copy()
        for s, v in zip(sites, newv):
            tgt = tgt + (v.astype(np.int64) - S[:, s].astype(np.int64)) * pw[s]
        rows.append(codes[nz]); cols.append(tgt[nz]); vals.append(c[nz])
    r = np.concatenate(rows) if rows else np.zeros(0, np.int64)
    cc = np.concatenate(cols) if cols else np.zeros(0, np.int64)
    v = np.concatenate(vals) if vals else np.zeros(0)
    Q = sp.coo_matrix((v, (r, cc)), shape=(nstate, nstate)).tocsr()
    Q = Q - sp.diags(np.asarray(Q.sum(axis=1)).ravel())
    return Q.tocsr()


def evolve(p, Q, t):
    """p e^{tQ} for a row vector p."""
    if t == 0:
        return p.copy()
    return expm_multiply(Q.T.tocsc() * t, p)


def lie(p, QE, QO, dt, n):
    for _ in range(n):
        p = evolve(evolve(p, QE, dt), QO, dt)
    return p


def strang(p, QE, QO, dt, n):
    for _ in range(n):
        p = evolve(evolve(evolve(p, QE, dt / 2), QO, dt), QE, dt / 2)
    return p


def random_sl_mean(p, QE, QO, dt, n):
    """Mean law of the sub-lattice random schedule: 2n windows of length dt,
    each E or O with probability 1/2 (Eq. SLPCS)."""
    for _ in range(2 * n):
        p = 0.5 * (evolve(p, QE, dt) + evolve(p, QO, dt))
    return p


def random_order_mean(p, QE, QO, dt, n):
    """Mean law of the random-order schedule: per step E then O or O then E."""
    for _ in range(n):
        p = 0.5 * (evolve(evolve(p, QE, dt), QO, dt) + evolve(evolve(p, QO, dt), QE, dt))
    return p


def point_mass(lx, ly, base, lattice):
    pw = base ** np.arange(lx * ly, dtype=np.int64)
    p = np.zeros(base ** (lx * ly))
    p[int(np.asarray(lattice, np.int64).reshape(-1) @ pw)] = 1.0
    return p


def codes_of(lattices, base):
    lat = np.asarray(lattices, np.int64)
    pw = base ** np.arange(lat.shape[1], dtype=np.int64)
    return lat @ pw


def gibbs_ising(lx, ly, betaJ):
    """Gibbs weights exp(-beta H) with H = -K sum_<xy> s_x s_y + h sum s_x,
    K = 4J, h = 2K (lattice-gas form of the zero-field Ising model)."""
    S = decode(lx, ly, 2).astype(np.float64)
    N = lx * ly
    pair = np.zeros(len(S))
    for i in range(N):
        for d in (1, 2):  # E and S: each bond once
            pair += S[:, i] * S[:, _nb(lx, ly, i, d)]
    bK, bh = 4.0 * betaJ, 8.0 * betaJ
    logw = bK * pair - bh * S.sum(axis=1)
    w = np.exp(logw - logw.max())
    return w / w.sum()


def gibbs_ising1d(lx, betaK, betah, ka=1.0, kd=1.0):
    """Stationary weights of the ring's adsorption/desorption dynamics:
    pi(s) proportional to (ka/kd)^N1 exp(beta K sum_x s_x s_{x+1} - beta h N1)
    (detailed balance of the ISING1D rates, written per configuration)."""
    S = decode(lx, 1, 2).astype(np.float64)
    pair = sum(S[:, i] * S[:, (i + 1) % lx] for i in range(lx))
    n1 = S.sum(axis=1)
    logw = betaK * pair + (np.log(ka / kd) - betah) * n1
    w = np.exp(logw - logw.max())
    return w / w.sum()


def window_frozen_halo(lx, ly, qx, qy, model, rates, snapshot, colour, h, cell):
    """Exact law of one cell's write set after a window of length h under the
    frozen-halo rule: the write set evolves by the cell's owned events, rates
    read from the write set's current values and, outside it, from the
    snapshot. Returns (write_set_sites, probabilities over write-set codes)."""
    ncx = lx // qx
    cx, cy = cell % ncx, cell // ncx
    X0, Y0 = cx * qx, cy * qy
    ws = [((Y0 + ly_) % ly) * lx + (X0 + lx_) % lx for ly_ in range(qy) for lx_ in range(qx)]
    if model in ("DIFFUSION", "ZGB"):
        if colour == 0:
            for ly_ in range(qy):
                ws.append(((Y0 + ly_) % ly) * lx + (X0 - 1) % lx)
                ws.append(((Y0 + ly_) % ly) * lx + (X0 + qx) % lx)
        else:
            for lx_ in range(qx):
                ws.append(((Y0 - 1) % ly) * lx + (X0 + lx_) % lx)
                ws.append(((Y0 + qy) % ly) * lx + (X0 + lx_) % lx)
    base = 3 if model == "ZGB" else 2
    snap = np.asarray(snapshot, np.int8).reshape(-1)
    nws = len(ws)
    local = decode(1, nws, base) if nws else np.zeros((1, 0), np.int8)
    # full configurations: snapshot with the write set replaced
    full = np.repeat(snap[None, :], len(local), axis=0)
    full[:, ws] = local
    own = set(ws[: qx * qy])
    _, _, evs = events(lx, ly, model, rates, full)
    pw = base ** np.arange(nws, dtype=np.int64)
    codes = local.astype(np.int64) @ pw
    pos = {s: k for k, s in enumerate(ws)}
    rows, cols, vals = [], [], []
    for owner, sites, newv, c in evs:
        if owner_colour(lx, ly, qx, qy, owner) != colour:
            continue
        if owner[0] == "site" and owner[1] not in own:
            continue
        if owner[0] == "bond":
            i, d = owner[1], owner[2]
            j = _nb(lx, ly, i, d)
            if i not in own and j not in own:
                continue
        tgt = codes.copy()
        for s, v in zip(sites, newv):
            tgt = tgt + (v.astype(np.int64) - full[:, s].astype(np.int64)) * pw[pos[s]]
        nz = c > 0
        rows.append(codes[nz]); cols.append(tgt[nz]); vals.append(c[nz])
    n = len(local)
    Q = sp.coo_matrix((np.concatenate(vals), (np.concatenate(rows), np.concatenate(cols))),
                      shape=(n, n)).tocsr()
    Q = Q - sp.diags(np.asarray(Q.sum(axis=1)).ravel())
    p0 = np.zeros(n)
    p0[int(snap[ws].astype(np.int64) @ pw)] = 1.0
    return ws, evolve(p0, Q.tocsr(), h)


def nested_colours(lx, ly, Qx, Qy, qx, qy, i):
    """(super-cell colour, sub-cell colour) of site i in the two-level
    checkerboard of Eq. sublatt2: super-cells Qx x Qy coloured by
    (cx + cy) mod 2, and inside each super-cell the sub-cells qx x qy coloured
    by their position within it."""
    x, y = i % lx, i // lx
    C = ((x // Qx) + (y // Qy)) % 2
    c = (((x % Qx) // qx) + ((y % Qy) // qy)) % 2
    return C, c


def generator_nested(lx, ly, Qx, Qy, qx, qy, model, rates, C, c):
    """Sparse generator of the site events of one (super colour, sub colour)
    part of Eq. opdecomp2 (spin-flip models: every event is a site event)."""
    S, base, evs = events(lx, ly, model, rates)
    assert model in ("ADSDES", "ISING")
    nstate = len(S)
    pw = base ** np.arange(lx * ly, dtype=np.int64)
    codes = S.astype(np.int64) @ pw
    rows, cols, vals = [], [], []
    for owner, sites, newv, cv in evs:
        if nested_colours(lx, ly, Qx, Qy, qx, qy, owner[1]) != (C, c):
            continue
        nz = cv > 0
        tgt = codes + (newv[0].astype(np.int64) - S[:, sites[0]].astype(np.int64)) * pw[sites[0]]
        rows.append(codes[nz]); cols.append(tgt[nz]); vals.append(cv[nz])
    Q = sp.coo_matrix((np.concatenate(vals), (np.concatenate(rows), np.concatenate(cols))),
                      shape=(nstate, nstate)).tocsr()
    Q = Q - sp.diags(np.asarray(Q.sum(axis=1)).ravel())
    return Q.tocsr()


def nested_window(p, QC, h, inner, n_in):
    """One outer window of length h of one super-cell colour: n_in inner
    steps of the inner splitting over its two sub-cell colours QC = (Q_C0,
    Q_C1) -- Lie: e^{d Q_C0} e^{d Q_C1}; Strang: e^{d/2 Q_C0} e^{d Q_C1}
    e^{d/2 Q_C0}; d = h / n_in."""
    d = h / n_in
    for _ in range(n_in):
        if inner == "LIE":
            p = evolve(evolve(p, QC[0], d), QC[1], d)
        else:
            p = evolve(evolve(evolve(p, QC[0], d / 2), QC[1], d), QC[0], d / 2)
    return p


def nested_product(p, Qs, scheme, dt, n, inner, n_in):
    """Law after n outer steps of the nested scheme (Eq. opdecomp2 composed
    by Eq. lie or Eq. strang at both levels). Qs[C][c] is the generator of
    super colour C, sub colour c."""
    for _ in range(n):
        if scheme == "LIE":
            p = nested_window(p, Qs[0], dt, inner, n_in)
            p = nested_window(p, Qs[1], dt, inner, n_in)
        else:
            p = nested_window(p, Qs[0], dt / 2, inner, n_in)
            p = nested_window(p, Qs[1], dt, inner, n_in)
            p = nested_window(p, Qs[0], dt / 2, inner, n_in)
    return p
