"""All-pairs / all-triples brute force of the swap potential for tiny systems.

Independent of ``oracle/``: no cell list, no neighbour list, no pair
bookkeeping -- every unordered pair and every (centre, unordered pair of
partners) triple of the system is visited with plain Python loops.  It pins the
oracle's list, triplet and periodic-image bookkeeping (the formulas themselves
are pinned by the closed forms of the paper in ``test_oracle_pins.py``).
"""
import math

import numpy as np


def _wrap(d, L):
    if d > 0.5 * L:
        return d - L
    if d < -0.5 * L:
        return d + L
    return d


def _box_fraction(x, L):
    """32-bit fraction of coordinate x along an edge L (FP32 decisions): the
    edge rounded to float and to the 2^-48 grid (Lq units), x wrapped into it
    and rounded half-even to the grid (q), then floor(q floor(2^96 / Lq) / 2^64)."""
    Lq = math.floor(float(np.float32(L)) * 2.0 ** 48 + 0.5)
    Lp = Lq * 2.0 ** -48
    k = math.floor(x / Lp)
    xw = x - k * Lp
    q = round(xw * 2.0 ** 48)  # Python rounds halves to even
    if q >= Lq:
        q -= Lq
    if q < 0:
        q += Lq
    return (q * ((1 << 96) // Lq)) >> 64, Lq


def _d2_decision(xi, xj, box, fp32):
    if fp32:
        f = np.float32
        acc = []
        for c in range(3):
            ui, Lq = _box_fraction(xi[c], box[c])
            uj, _ = _box_fraction(xj[c], box[c])
            du = ((uj - ui + 2 ** 31) % 2 ** 32) - 2 ** 31  # signed 32-bit wrap: the minimum image
            acc.append(f(du) * f(Lq * 2.0 ** -80))
        s = acc[0] * acc[0]
        s = s + acc[1] * acc[1]
        s = s + acc[2] * acc[2]
        return float(s)
    acc = [_wrap(xj[c] - xi[c], box[c]) for c in range(3)]
    return (acc[0] * acc[0] + acc[1] * acc[1]) + acc[2] * acc[2]


def _cut2(c, fp32):
    return float(np.float32(c * c)) if fp32 else c * c


def _lj(r, eps, sig, n):
    x = (sig / r) ** n
    return 4 * eps * (x * x - x), 4 * eps * (-2 * n * x * x + n * x) / r


def brute(x, types, pairs, box, fp32=False):
    """pairs: {(ti, tj): dict(kind, eps, sigma, n, rcut, lambda3, shift, rbond)}."""
    x = np.asarray(x, dtype=np.float64)
    n = len(x)

    def par(ti, tj):
        return pairs.get((ti, tj)) or pairs.get((tj, ti)) or {"kind": 0}

    def rmin(p):
        return p["sigma"] * 2.0 ** (1.0 / p["n"])

    def vec(i, j):  # x_i - x_j, minimum image
        return np.array([_wrap(x[i, c] - x[j, c], box[c]) for c in range(3)])

    def inside(i, j):
        p = par(types[i], types[j])
        if p["kind"] == 1:
            c = rmin(p)
        elif p["kind"] == 2:
            c = p["rcut"]
        else:
            return False
        return _d2_decision(x[i], x[j], box, fp32) < _cut2(c, fp32)

    def vhat(p, r):
        if r <= rmin(p):
            return 1.0, 0.0
        vc = _lj(p["rcut"], p["eps"], p["sigma"], p["n"])[0] if p.get("shift", 0) else 0.0
        v, dv = _lj(r, p["eps"], p["sigma"], p["n"])
        den = p["eps"] + vc
        return (vc - v) / den, -dv / den

    F = np.zeros((n, 3))
    U2 = U3 = 0.0
    W = np.zeros((3, 3))
    nb = 0
    for i in range(n):
        for j in range(i + 1, n):
            if not inside(i, j):
                continue
            p = par(types[i], types[j])
            d = vec(i, j)
            r = math.sqrt(d @ d)
            v, dv = _lj(r, p["eps"], p["sigma"], p["n"])
            if p["kind"] == 1:
                u = v + p["eps"]
            else:
                vc = _lj(p["rcut"], p["eps"], p["sigma"], p["n"])[0] if p.get("shift", 0) else 0.0
                u = v - vc
                if _d2_decision(x[i], x[j], box, fp32) < _cut2(p["rbond"], fp32):
                    nb += 1
            U2 += u
            f = -dv / r * d
            F[i] += f
            F[j] -= f
            W += np.outer(d, f)
    for i in range(n):
        for j in range(n):
            for k in range(j + 1, n):
                if i in (j, k):
                    continue
                pj, pk = par(types[i], types[j]), par(types[i], types[k])
                if pj["kind"] != 2 or pk["kind"] != 2:
                    continue
                if not (inside(i, j) and inside(i, k)):
                    continue
                dj, dk = vec(i, j), vec(i, k)
                rj, rk = math.sqrt(dj @ dj), math.sqrt(dk @ dk)
                hj, dhj = vhat(pj, rj)
                hk, dhk = vhat(pk, rk)
                a = math.sqrt(pj["lambda3"] * pj["eps"]) * math.sqrt(pk["lambda3"] * pk["eps"])
                U3 += a * hj * hk
                fj = -a * dhj * hk / rj * dj
                fk = -a * hj * dhk / rk * dk
                F[i] += fj + fk
                F[j] -= fj
                F[k] -= fk
                W += np.outer(dj, fj) + np.outer(dk, fk)
    Wv = np.array([W[0, 0], W[1, 1], W[2, 2], W[0, 1], W[0, 2], W[1, 2]])
    return dict(U2=U2, U3=U3, F=F, W=Wv, n_bonds=nb)


def brute_nlist(x, types, pairs, box, skin, fp32=False):
    """Sorted neighbour sets within r_cut(ti, tj) + skin for every particle."""
    n = len(x)
    out = [[] for _ in range(n)]
    for i in range(n):
        for j in range(n):
            if i == j:
                continue
            p = pairs.get((types[i], types[j])) or pairs.get((types[j], types[i])) or {"kind": 0}
            if p["kind"] == 1:
                c = p["sigma"] * 2.0 ** (1.0 / p["n"])
            elif p["kind"] == 2:
                c = p["rcut"]
            else:
                continue
            if _d2_decision(x[i], x[j], box, fp32) < _cut2(c + skin, fp32):
                out[i].append(j)
    return [np.array(sorted(o), dtype=np.int64) for o in out]
