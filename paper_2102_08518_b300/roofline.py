"""Algorithmic memory work of a stencil gather, for roofline accounting.

For random points the coefficient gathers of one point touch a set of 32-byte
sectors that no layout-preserving kernel can avoid fetching; their number
(per point, averaged over a sample) is the algorithmic sector traffic the
gather roofline is measured in.  Computed here from the sub-region table with
the same region of evaluation, folding and storage layout the kernels use.
"""
from __future__ import annotations

import numpy as np


def shift_masks(kernel_source: str):
    """The copy-choice masks (x, y) a generated kernel for the shifted bricked
    copies carries (see the generator's shift_rule)."""
    import re
    m = re.findall(r"const int s([xyz]) = \(int\)\(\((\d+)ull >> ", kernel_source)
    d = {k: int(v) for k, v in m}
    return tuple(d[a] for a in "xyz" if a in d)


def stencil_indices(table, ext, pts: np.ndarray, layout: str = "coset", masks=None) -> np.ndarray:
    """Linear coefficient indices (n_points, n_sites) of every point's stencil
    in the volume layout ("coset": coset j's array after array j - 1;
    "interleaved": the cosets' values of one grid index adjacent; "bricked":
    2 x 2 x 2 bricks of grid indices with the cosets adjacent inside;
    "bricked_shifted": the four shifted bricked copies, each point in the copy
    the kernel's copy-choice masks pick); -1 where a site lies outside the
    arrays."""
    spl = table.spline
    lat = spl.lattice
    D = lat.dim
    e = np.array(list(ext)[:D], dtype=np.int64)
    x = pts.astype(np.float32).astype(np.float64)
    n = len(x)
    # region of evaluation
    if spl.roe == "parallelepiped":
        k = np.floor(x)
    else:
        best = None
        for l in lat.cosets:
            l = np.asarray(l[:D], dtype=np.float64)
            kk = lat.scale * np.round((x - l) / lat.scale) + l
            d = np.sum((x - kk) ** 2, axis=1)
            if best is None:
                best, k = d, kk
            else:
                sel = d < best
                best = np.where(sel, d, best)
                k = np.where(sel[:, None], kk, k)
    y = x - k
    k = k.astype(np.int64)
    if table.fold == "hyperoctahedral":
        a = np.abs(y)
        order = np.argsort(-a, axis=1, kind="stable")
        sign = np.where(y < 0, -1, 1)
        yref = np.take_along_axis(a, order, axis=1)
    else:
        order = np.tile(np.arange(D), (n, 1))
        sign = np.ones((n, D), dtype=np.int64)
        yref = y
    regions = np.array([table.region_of(r) for r in yref]) if len(table.regions) > 1 else np.zeros(n, int)
    shift = np.zeros((n, 3), dtype=np.int64)
    if layout in ("bricked_shifted", "bricked_shifted_xyz"):
        for i, mask in enumerate(masks):
            if table.fold == "hyperoctahedral":
                r_i = np.argmax(order == i, axis=1)
                neg = (sign[:, i] < 0).astype(np.int64)
            else:
                r_i = np.full(n, i)
                neg = np.zeros(n, dtype=np.int64)
            psi = regions if len(table.regions) <= 2 else np.zeros_like(regions)
            key = ((psi * 3 + r_i) * 2 + neg) * 4 + (k[:, i] & 3)
            shift[:, i] = (np.array([mask >> int(q) for q in key], dtype=object) & 1).astype(np.int64)
    nsite = max(len(r.sites) for r in table.regions)
    out = np.full((n, nsite), -1, dtype=np.int64)
    per = int(np.prod(e))
    lut = np.full(2 ** D, -1, dtype=np.int64)
    for j, l in enumerate(lat.cosets):
        lut[sum(((v % 2) << i) for i, v in enumerate(l[:D]))] = j
    for ri, reg in enumerate(table.regions):
        m = regions == ri
        if not np.any(m):
            continue
        for j, s in enumerate(reg.sites):
            off = np.zeros((int(m.sum()), D), dtype=np.int64)
            for r in range(D):
                cart = order[m, r]
                off[np.arange(len(cart)), cart] = sign[m][np.arange(len(cart)), cart] * s[r]
            nn = k[m] + off
            if lat.scale == 2:
                cid = lut[np.sum((nn & 1) << np.arange(D), axis=1)]
                idx = nn >> 1
            else:
                cid = np.zeros(len(nn), dtype=np.int64)
                idx = nn
            ok = np.all((idx >= 0) & (idx < e), axis=1)
            q = idx[:, 0] + e[0] * (idx[:, 1] + (e[1] * idx[:, 2] if D == 3 else 0))
            C = len(lat.cosets)
            if layout == "bricked":
                i2 = idx[:, 2] if D == 3 else np.zeros_like(idx[:, 0])
                bk = idx[:, 0] // 2 + (e[0] // 2) * (idx[:, 1] // 2 + (e[1] // 2) * (i2 // 2))
                w = idx[:, 0] % 2 + 2 * (idx[:, 1] % 2) + 4 * (i2 % 2)
                lin = (bk * (8 if D == 3 else 4) + w) * C + cid
            elif layout in ("bricked_shifted", "bricked_shifted_xyz"):
                sh = shift[m]
                pz = 2 if layout == "bricked_shifted_xyz" else 0
                j0, j1, j2 = idx[:, 0] + sh[:, 0], idx[:, 1] + sh[:, 1], idx[:, 2] + sh[:, 2]
                bk = j0 // 2 + ((e[0] + 2) // 2) * (j1 // 2 + ((e[1] + 2) // 2) * (j2 // 2))
                w = j0 % 2 + 2 * (j1 % 2) + 4 * (j2 % 2)
                copy = C * (e[0] + 2) * (e[1] + 2) * (e[2] + pz)
                lin = (sh[:, 0] + 2 * sh[:, 1] + 4 * sh[:, 2]) * copy + (bk * 8 + w) * C + cid
            elif layout == "interleaved":
                lin = q * C + cid
            else:
                lin = q + cid * per
            out[np.where(m)[0], j] = np.where(ok, lin, -1)
    return out


def distinct_sectors_per_point(table, ext, pts: np.ndarray, elem_bytes: int = 4, layout: str = "coset",
                               masks=None) -> float:
    idx = stencil_indices(table, ext, pts, layout, masks)
    sec = np.where(idx >= 0, (idx * elem_bytes) // 32, -1)
    sec.sort(axis=1)
    distinct = (np.diff(sec, axis=1) != 0).sum(axis=1) + 1 - (sec[:, 0] < 0)
    return float(distinct.mean())


def distinct_lines_per_point(table, ext, pts: np.ndarray, elem_bytes: int = 4, layout: str = "coset") -> float:
    """Distinct 128-byte cache lines of one point's stencil (L1 allocates lines)."""
    idx = stencil_indices(table, ext, pts, layout)
    sec = np.where(idx >= 0, (idx * elem_bytes) // 128, -1)
    sec.sort(axis=1)
    distinct = (np.diff(sec, axis=1) != 0).sum(axis=1) + 1 - (sec[:, 0] < 0)
    return float(distinct.mean())


def tensor_shape(table, expansion: str = "sparse", kstep: int = 8):
    """Shape of the coefficient-transform product of the tensor-core value
    kernel: K = union stencil sites rounded up to kstep (8: the TF32 product's K
    step; 16: the FP16 form's),
    N = the (region, monomial) columns with a nonzero entry rounded up to 16
    (at least 16), and the nonzero count of the transform matrix (the FMA
    path's multiply-adds).  Returns (K, N, nnz)."""
    regions = table.regions_centroid if expansion == "centroid" and table.regions_centroid else table.regions
    union = []
    for r in regions:
        for s in r.sites:
            if tuple(s) not in union:
                union.append(tuple(s))
    ncol, nnz = 0, 0
    for r in regions:
        M = r.coef_matrix()
        for a in range(len(r.monomials)):
            col = sum(1 for j in range(len(r.sites)) if M[j][a] != 0)
            if col:
                ncol += 1
                nnz += col
    K = (len(union) + kstep - 1) // kstep * kstep
    N = max(16, (ncol + 15) // 16 * 16)
    return K, N, nnz


def case_roofline(fma_per_point: int, coef_bytes_per_point: float, n: int, ms: float, sms: int, sm_mhz: float,
                  l2_gbs: float, hbm_gbs: float, stream_bytes_per_point: float = 16.0) -> dict:
    """Roofline of one evaluation launch over n points taking ms milliseconds.

    Two roofs bound it: the FP32 FMA pipe for the generated kernel's
    multiply-adds (fma_per_point; SMs x 128 FMA lanes per clock at the observed
    SM clock), and the gathers: the point's coefficient bytes at the rate the
    level they come from (L2 for a resident volume) delivers them, plus the
    point stream (coordinates in, value out) at the HBM rate.  The binding roof
    is the slower one; frac = its time / the measured time."""
    t_fma = fma_per_point * n / (sms * 128.0 * sm_mhz * 1e6) * 1e3
    t_gather = (coef_bytes_per_point * n / (l2_gbs * 1e9) + stream_bytes_per_point * n / (hbm_gbs * 1e9)) * 1e3
    alu = t_fma >= t_gather
    t_roof = t_fma if alu else t_gather
    out = {"bound": "alu" if alu else "l2", "ms": round(ms, 4), "t_fma_ms": round(t_fma, 4),
           "t_gather_ms": round(t_gather, 4), "frac": round(t_roof / ms, 4)}
    if alu:
        out.update(unit="TFLOP/s", achieved=round(2.0 * fma_per_point * n / (ms * 1e-3) / 1e12, 2),
                   peak=round(2.0 * sms * 128.0 * sm_mhz * 1e6 / 1e12, 2))
    else:
        per_pt = coef_bytes_per_point + stream_bytes_per_point
        out.update(unit="GB/s", achieved=round(per_pt * n / (ms * 1e-3) / 1e9, 1),
                   peak=round(per_pt * n / (t_gather * 1e-3) / 1e9, 1))
    return out
