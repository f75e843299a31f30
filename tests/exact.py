"""Exact results used to pin the CPU oracle.  Nothing here calls the oracle.

* Brute-force Boltzmann averages on tiny periodic lattices (Ising, Potts
  Eq. 1, clock Eq. clock of Komura & Okabe, arXiv:1202.0635).
* The exact one-step Swendsen-Wang transition row from a given
  configuration, by enumerating every subset of the bonds that can form
  (Sec. 2 steps (i)-(vii); clock: Sec. 4 embedded clusters).
* Kaufman's exact partition function of the L x L Ising torus, giving the
  exact finite-size energy (Onsager's value -sqrt(2) per site at Tc in the
  L -> infinity limit).
* Statistics helpers (binned error bars, chi-square).
"""
import math

import numpy as np


def torus_bonds(L):
    """(a, b) pairs of every bond: site i=y*L+x to its right and down neighbour."""
    out = []
    for y in range(L):
        for x in range(L):
            i = y * L + x
            out.append((i, y * L + (x + 1) % L))
            out.append((i, ((y + 1) % L) * L + x))
    return np.array(out, dtype=np.int64)


def all_states(N, q):
    """Every configuration of N sites with q states: shape (q**N, N) int8."""
    grids = np.indices((q,) * N, dtype=np.int8).reshape(N, -1).T
    return np.ascontiguousarray(grids)


def _boltzmann(E, beta):
    w = np.exp(-beta * (E - E.min()))
    return w / w.sum()


def ising_exact(L, T):
    """Exact <E/N>, <|m|>, <m^2>, <m^4> of the Ising torus, H = -sum s_i s_j."""
    N = L * L
    b = torus_bonds(L)
    s = 1 - 2 * all_states(N, 2).astype(np.int64)          # state 0 -> +1
    E = -(s[:, b[:, 0]] * s[:, b[:, 1]]).sum(axis=1).astype(np.float64)
    m = s.sum(axis=1) / N
    w = _boltzmann(E, 1.0 / T)
    return {"e": float(w @ E) / N, "absm": float(w @ np.abs(m)),
            "m2": float(w @ m ** 2), "m4": float(w @ m ** 4)}


def ising_correlation_exact(L, T, r):
    """Exact <s_i s_{i+r}> of the Ising torus (H = -sum s_i s_j), averaged over
    every site and both lattice directions."""
    N = L * L
    s = 1 - 2 * all_states(N, 2).astype(np.int64)
    b = torus_bonds(L)
    E = -(s[:, b[:, 0]] * s[:, b[:, 1]]).sum(axis=1).astype(np.float64)
    idx = np.arange(N).reshape(L, L)
    px = np.roll(idx, -r, axis=1).reshape(-1)   # site (y, x + r)
    py = np.roll(idx, -r, axis=0).reshape(-1)   # site (y + r, x)
    c = ((s * s[:, px]).sum(axis=1) + (s * s[:, py]).sum(axis=1)) / (2.0 * N)
    w = _boltzmann(E, 1.0 / T)
    return float(w @ c)


def potts_exact(L, q, T):
    """Exact <E/N>, <m^2> of the q-state Potts torus, Eq. (1): E = #unequal pairs,
    m^2 = M^2/N^2 with M^2 from Eq. (M^2)."""
    N = L * L
    b = torus_bonds(L)
    s = all_states(N, q)
    E = (s[:, b[:, 0]] != s[:, b[:, 1]]).sum(axis=1).astype(np.float64)
    n = np.stack([(s == k).sum(axis=1) for k in range(q)], axis=1).astype(np.float64)
    M2 = (q * (n ** 2).sum(axis=1) - N * N) / (q - 1)
    w = _boltzmann(E, 1.0 / T)
    return {"e": float(w @ E) / N, "m2": float(w @ M2) / N ** 2}


def clock_exact(L, q, T, chunk=1 << 20):
    """Exact <E/N>, <m^2> of the q-state clock torus, H = -sum cos(th_i - th_j)."""
    N = L * L
    b = torus_bonds(L)
    cosd = np.cos(2 * np.pi * np.arange(q) / q)
    sind = np.sin(2 * np.pi * np.arange(q) / q)
    total = q ** N
    Es, M2s = [], []
    for start in range(0, total, chunk):
        idx = np.arange(start, min(total, start + chunk), dtype=np.int64)
        s = np.empty((idx.size, N), dtype=np.int64)
        r = idx.copy()
        for k in range(N - 1, -1, -1):
            s[:, k] = r % q
            r //= q
        d = (s[:, b[:, 0]] - s[:, b[:, 1]]) % q
        Es.append(-cosd[d].sum(axis=1))
        M2s.append(cosd[s].sum(axis=1) ** 2 + sind[s].sum(axis=1) ** 2)
    E = np.concatenate(Es)
    M2 = np.concatenate(M2s)
    w = _boltzmann(E, 1.0 / T)
    return {"e": float(w @ E) / N, "m2": float(w @ M2) / N ** 2}


def components_of_subsets(N, bonds, masks):
    """Min-site-index component labels for many bond subsets at once.

    bonds: (B, 2) site pairs; masks: (S,) integers, bit k = bond k present.
    Returns (S, N) int64 labels.  Plain label propagation to a fixed point.
    """
    S = masks.size
    lab = np.tile(np.arange(N, dtype=np.int64), (S, 1))
    present = [((masks >> k) & 1).astype(bool) for k in range(len(bonds))]
    while True:
        changed = False
        for k, (a, c) in enumerate(bonds):
            p = present[k]
            m = np.minimum(lab[:, a], lab[:, c])
            upd = p & ((lab[:, a] != m) | (lab[:, c] != m))
            if upd.any():
                changed = True
                lab[upd, a] = m[upd]
                lab[upd, c] = m[upd]
        if not changed:
            return lab


def potts_bond_p(K):
    """Sec. 2 step (ii): a bond forms between equal states with p = 1 - e^{-K}."""
    p = -math.expm1(-K)
    return lambda sa, sb: p if sa == sb else 0.0


def clock_bond_p(q, K, axis):
    """Embedded Ising bond of the clock model for mirror axis angle pi*axis/q:
    with projections s = sin(theta - pi*axis/q) the bond forms only when
    s_a s_b > 0, with p = 1 - exp(-2 K s_a s_b) (Wolff's embedding)."""
    def proj(k):
        j = (2 * k - axis) % (2 * q)
        if j % q == 0:
            return 0.0
        return math.sin(math.pi * j / q)

    def p(sa, sb):
        x = proj(sa) * proj(sb)
        return -math.expm1(-2.0 * K * x) if x > 0 else 0.0
    return p


def sw_transition_row(L, q, model, sigma, bond_p, axis=None):
    """Exact one-sweep transition probabilities out of configuration sigma.

    Every bond (a, b) forms independently with probability
    bond_p(sigma_a, sigma_b).  model 'potts': every cluster then takes each
    of q states with probability 1/q.  model 'clock' (mirror axis index m):
    every cluster is reflected, k -> (m - k) mod q, with probability 1/2.
    Returns (codes, probs): sorted integer codes (see encode) of every
    reachable sigma' and their exact probabilities.
    """
    N = L * L
    sigma = np.asarray(sigma, dtype=np.int64).reshape(-1)
    bonds = torus_bonds(L)
    probs = []
    live = []
    for k, (a, c) in enumerate(bonds):
        pk = bond_p(int(sigma[a]), int(sigma[c]))
        if pk > 0:
            live.append((a, c))
            probs.append(pk)
    live = np.array(live, dtype=np.int64).reshape(-1, 2)
    nb = len(live)
    masks = np.arange(1 << nb, dtype=np.int64)
    w = np.ones(masks.size)
    for k in range(nb):
        bit = ((masks >> k) & 1).astype(bool)
        w *= np.where(bit, probs[k], 1.0 - probs[k])
    lab = components_of_subsets(N, live, masks)
    # group the subsets by the partition they induce
    part, inv = np.unique(lab, axis=0, return_inverse=True)
    pw = np.zeros(part.shape[0])
    np.add.at(pw, inv.reshape(-1), w)
    all_codes, all_p = [], []
    for p, weight in zip(part, pw):
        roots, site_cluster = np.unique(p, return_inverse=True)
        nc = roots.size
        if model == "clock":
            choice = all_states(nc, 2).astype(np.int64)           # 1 = reflect
            ch = choice[:, site_cluster]
            new = np.where(ch == 1, (axis - sigma[None, :]) % q, sigma[None, :])
            prob = weight / 2.0 ** nc
        else:
            choice = all_states(nc, q).astype(np.int64)
            new = choice[:, site_cluster]
            prob = weight / float(q) ** nc
        all_codes.append(encode(new, q))
        all_p.append(np.full(new.shape[0], prob))
    codes, inv = np.unique(np.concatenate(all_codes), return_inverse=True)
    probs = np.zeros(codes.size)
    np.add.at(probs, inv, np.concatenate(all_p))
    return codes, probs


def encode(states, q):
    """Configuration(s) -> integer code in base q, site 0 most significant."""
    s = np.atleast_2d(np.asarray(states, dtype=np.int64))
    code = np.zeros(s.shape[0], dtype=np.int64)
    for k in range(s.shape[1]):
        code = code * q + s[:, k]
    return code


def chi2_pvalue(sample_codes, codes, probs, min_expected=5.0):
    """Pearson chi-square p-value of sampled codes against exact probabilities.

    Categories with expected count below min_expected are pooled.  Returns
    (p_value, n_impossible) where n_impossible counts samples that fell on
    a configuration of zero exact probability."""
    from scipy import stats
    M = sample_codes.size
    idx = np.searchsorted(codes, sample_codes)
    idx = np.clip(idx, 0, codes.size - 1)
    hit = codes[idx] == sample_codes
    n_impossible = int((~hit).sum())
    obs = np.bincount(idx[hit], minlength=codes.size).astype(np.float64)
    exp = probs * M
    big = exp >= min_expected
    o = list(obs[big])
    e = list(exp[big])
    if (~big).any():
        o.append(obs[~big].sum())
        e.append(exp[~big].sum())
    o, e = np.array(o), np.array(e)
    e *= o.sum() / e.sum()
    return float(stats.chisquare(o, e).pvalue), n_impossible


def kaufman_lnZ(L, K, mp):
    """ln Z of the L x L Ising torus (H = -sum s_i s_j, K = 1/T), Kaufman 1949.

    Z = 1/2 (2 sinh 2K)^(N/2) (Z1 + Z2 + Z3 + Z4) with
      Z1 = prod_r 2 cosh(L g_{2r+1} / 2),  Z2 = prod_r 2 sinh(L g_{2r+1} / 2),
      Z3 = prod_r 2 cosh(L g_{2r} / 2),    Z4 = prod_r 2 sinh(L g_{2r} / 2),
    r = 0 .. L-1, cosh g_l = cosh 2K coth 2K - cos(pi l / L) for l >= 1 and
    g_0 = 2K + ln tanh K (negative above Tc, which makes Z4 change sign).
    """
    K = mp.mpf(K)
    c = mp.cosh(2 * K) * mp.coth(2 * K)

    def g(l):
        if l == 0:
            return 2 * K + mp.log(mp.tanh(K))
        return mp.acosh(c - mp.cos(mp.pi * l / L))

    z1 = z2 = z3 = z4 = mp.mpf(1)
    for r in range(L):
        go, ge = g(2 * r + 1), g(2 * r)
        z1 *= 2 * mp.cosh(L * go / 2)
        z2 *= 2 * mp.sinh(L * go / 2)
        z3 *= 2 * mp.cosh(L * ge / 2)
        z4 *= 2 * mp.sinh(L * ge / 2)
    N = L * L
    return mp.log(mp.mpf(1) / 2) + (mp.mpf(N) / 2) * mp.log(2 * mp.sinh(2 * K)) + mp.log(z1 + z2 + z3 + z4)


def kaufman_energy(L, T, dps=60):
    """Exact <E>/N of the L x L Ising torus at temperature T (J = 1)."""
    import mpmath as mp
    mp.mp.dps = dps
    K = mp.mpf(1) / mp.mpf(T)
    dlnZ = mp.diff(lambda k: kaufman_lnZ(L, k, mp), K)
    return float(-dlnZ / (L * L))


def binned(x, nbins=50):
    """Mean and binned standard error of a time series."""
    x = np.asarray(x, dtype=np.float64)
    n = (x.size // nbins) * nbins
    b = x[:n].reshape(nbins, -1).mean(axis=1)
    return float(b.mean()), float(b.std(ddof=1) / math.sqrt(nbins))
