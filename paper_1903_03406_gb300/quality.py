"""Quality report of an exported mesh (host, numpy): dihedral angles and
radius-edge ratios.

This is a report over the output of cdr_export, not a step of the refinement:
the library never calls it. The quantities are those Sec. 1 and the
experiments judge an output by: the radius-edge ratio R / l_min that the bound
B caps (Sec. 1), and the distribution of dihedral angles between 0 and 180
degrees (Sec. 3, Fig. 2's histograms).
"""
from __future__ import annotations

import numpy as np

# the six edges of a tetrahedron (i, j) and, for each, the two vertices off it
# (k, l): the edge's dihedral angle is the one between faces opposite k and l
EDGES = ((0, 1), (0, 2), (0, 3), (1, 2), (1, 3), (2, 3))
_OFF = tuple(tuple(v for v in range(4) if v not in e) for e in EDGES)
# bin edges of the radius-edge histogram (0.6 to 3.0 by 0.1)
RHO_EDGES = np.round(np.arange(0.6, 3.0001, 0.1), 10)


def _corners(xyz, tets):
    xyz = np.asarray(xyz, dtype=np.float64).reshape(-1, 3)
    tets = np.asarray(tets, dtype=np.int64).reshape(-1, 4)
    return xyz[tets]  # (n, 4, 3)


def dihedral_angles(xyz, tets):
    """(n, 6) dihedral angles in degrees, at the edges in EDGES order (NaN for a
    flat tetrahedron).

    The face opposite vertex k has an outward normal n_k (its cross product,
    flipped to point away from vertex k). Two faces meeting at an edge form the
    interior angle pi - angle(n_k, n_l)."""
    P = _corners(xyz, tets)
    normals = []
    for k in range(4):
        f = [P[:, v] for v in range(4) if v != k]
        n = np.cross(f[1] - f[0], f[2] - f[0])
        away = np.einsum("ij,ij->i", n, f[0] - P[:, k])
        normals.append(np.where((away < 0)[:, None], -n, n))
    out = np.empty((len(P), 6))
    with np.errstate(invalid="ignore", divide="ignore"):
        for e, (k, l) in enumerate(_OFF):
            nk, nl = normals[k], normals[l]
            c = -np.einsum("ij,ij->i", nk, nl) / (np.linalg.norm(nk, axis=1) *
                                                   np.linalg.norm(nl, axis=1))
            out[:, e] = np.degrees(np.arccos(np.clip(c, -1.0, 1.0)))
    return out


def radius_edge(xyz, tets):
    """(n,) circumradius / shortest edge of each tetrahedron (Sec. 1's quality
    measure; inf for a flat one). With u, v, w the edges from vertex a, the
    circumcentre is a + (|u|^2 v x w + |v|^2 w x u + |w|^2 u x v) / (2 u . v x w)."""
    P = _corners(xyz, tets)
    a = P[:, 0]
    u, v, w = P[:, 1] - a, P[:, 2] - a, P[:, 3] - a
    sq = lambda x: np.einsum("ij,ij->i", x, x)[:, None]
    num = sq(u) * np.cross(v, w) + sq(v) * np.cross(w, u) + sq(w) * np.cross(u, v)
    det = 2.0 * np.einsum("ij,ij->i", u, np.cross(v, w))
    lmin = np.min([np.linalg.norm(P[:, i] - P[:, j], axis=1) for i, j in EDGES], axis=0)
    with np.errstate(invalid="ignore", divide="ignore"):
        R = np.linalg.norm(num / det[:, None], axis=1)
        rho = R / lmin
    return np.where(det != 0, rho, np.inf)


def report(xyz, tets, B=None, bin_deg=10.0):
    """Summary of a mesh's quality: dihedral-angle extremes and histogram
    (fractions per bin of bin_deg degrees over [0, 180]), and, when B is given,
    the fraction of tetrahedra with radius-edge ratio above B. Flat tetrahedra
    (none in a valid mesh) are counted apart and left out of the angles."""
    ang = dihedral_angles(xyz, tets)
    flat = ~np.all(np.isfinite(ang), axis=1)
    ang = ang[~flat].ravel()
    edges = np.arange(0.0, 180.0 + bin_deg / 2, bin_deg)
    hist, _ = np.histogram(ang, bins=edges)
    out = {
        "tets": int(len(flat)),
        "flat_tets": int(flat.sum()),
        "dihedral_min_deg": float(ang.min()) if len(ang) else None,
        "dihedral_max_deg": float(ang.max()) if len(ang) else None,
        "dihedral_bin_deg": bin_deg,
        "dihedral_hist": [float(h) for h in hist / max(len(ang), 1)],
    }
    if B is not None:
        rho = radius_edge(xyz, tets)
        out["radius_edge_max"] = float(rho.max()) if len(rho) else None
        out["frac_above_B"] = float(np.mean(rho > B)) if len(rho) else 0.0
        # the ratio's distribution: bins of 0.1 from sqrt(6)/4 (the regular
        # tetrahedron, the smallest possible value) rounded down to 0.6, the last
        # bin open-ended
        h, _ = np.histogram(np.minimum(rho, RHO_EDGES[-1] - 1e-9), bins=RHO_EDGES)
        out["radius_edge_bins"] = [float(x) for x in RHO_EDGES]
        out["radius_edge_hist"] = [float(x) for x in h / max(len(rho), 1)]
    return out


def hist_distance(h1, h2):
    """Total variation distance between two dihedral histograms (0 = equal, 1 = disjoint)."""
    return 0.5 * float(np.abs(np.asarray(h1) - np.asarray(h2)).sum())
