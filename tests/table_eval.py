"""FP64 CPU evaluation of a sub-region table by Algorithm 1 (test helper only).

Used to check the generated tables (region of evaluation, folding, BSP planes,
sigma, stencils, polynomials) against the oracle's naive sum on tiny inputs,
independently of the GPU.  Not part of the product.
"""
import numpy as np

import workloads


def _roe(table, x):
    spl = table.spline
    lat = spl.lattice
    if spl.roe == "parallelepiped":
        return np.floor(x)
    best, bk = None, None
    for l in lat.cosets:
        l = np.asarray(l, dtype=np.float64)
        k = lat.scale * np.round((x - l) / lat.scale) + l        # np.round: half to even
        d = np.sum((x - k) ** 2)
        if best is None or d < best:
            best, bk = d, k
    return bk


def eval_table(table, coef, ext, pts):
    """f at pts (n, dim) from the table; coef shaped like workloads' arrays."""
    spl = table.spline
    lat = spl.lattice
    D = lat.dim
    flat = np.asarray(coef, dtype=np.float64).ravel()
    e = list(ext) + [1] * (3 - len(ext))
    per = int(np.prod(e[:D]))
    out = np.zeros(len(pts))
    for q, x in enumerate(np.asarray(pts, dtype=np.float64)):
        k = _roe(table, x)
        y = x - k
        if table.fold == "hyperoctahedral":
            neg = y < 0
            a = np.abs(y)
            order = sorted(range(D), key=lambda i: -a[i])           # stable: ties keep axis order
            yref = a[order]
        else:
            order = list(range(D))
            neg = np.zeros(D, dtype=bool)
            yref = y
        r = table.region_of(yref)
        reg = table.regions[r]
        f = 0.0
        u = [yref[i] - float(reg.center[i]) for i in range(D)]
        for s, w in zip(reg.sites, reg.weights):
            m = np.zeros(D)
            for rr in range(D):
                m[order[rr]] = (-1 if neg[order[rr]] else 1) * s[rr]
            n = (k + m).astype(np.int64)
            j = lat.coset_of(tuple(int(v) for v in n))
            idx = (n - np.asarray(lat.cosets[j][:D])) // lat.scale
            if np.any(idx < 0) or np.any(idx >= np.asarray(e[:D])):
                continue
            lin = j * per + int(idx[0]) + e[0] * (int(idx[1]) + (e[1] * int(idx[2]) if D == 3 else 0))
            f += flat[lin] * w.evalf(u)
        out[q] = f
    return out


def eval_separable(table, coef, ext, pts):
    """f at pts from the per-axis factors of a tensor-product table (the form the
    generated kernels evaluate): product of 1D weights in u_i = y_i - centre."""
    spl = table.spline
    D = spl.lattice.dim
    flat = np.asarray(coef, dtype=np.float64).ravel()
    e = list(ext) + [1] * (3 - len(ext))
    out = np.zeros(len(pts))
    for q, x in enumerate(np.asarray(pts, dtype=np.float64)):
        k = _roe(table, x)
        y = x - k
        ws = []
        for i, ax in enumerate(table.separable):
            u = y[i] - float(ax.center)
            ws.append([(s, w.evalf([u])) for s, w in zip(ax.sites, ax.weights)])
        f = 0.0
        for combo in np.ndindex(*[len(w) for w in ws]):
            n = [int(k[i]) + ws[i][combo[i]][0] for i in range(D)]
            if any(n[i] < 0 or n[i] >= e[i] for i in range(D)):
                continue
            wt = np.prod([ws[i][combo[i]][1] for i in range(D)])
            lin = n[0] + e[0] * (n[1] + (e[1] * n[2] if D == 3 else 0))
            f += flat[lin] * wt
        out[q] = f
    return out
