"""Comparison helpers shared by the GPU parity tests (test code only)."""
import numpy as np

from paper_2609_29081_b300 import workloads as W


def component_scales(ref_sites, dim):
    """Scale of each conservative component over all DoF sites; the momentum
    components share one scale (same units). A component whose residual vanishes
    by symmetry (e.g. rho*v in a y-uniform flow) is then judged against the
    magnitude of the terms that cancel in it, not against its own roundoff."""
    nc = dim + 2
    s = np.array([max(np.abs(site[c]).max() for site in ref_sites) for c in range(nc)])
    mom = s[1:1 + dim].max()
    s[1:1 + dim] = mom
    return np.maximum(s, 1e-300)


def max_rel_err(got, ref, dim, n):
    """max over sites and components of |got - ref|_inf / scale_c."""
    gs = W.split_sites(got, dim, *n)
    rs = W.split_sites(ref, dim, *n)
    sc = component_scales(rs, dim)
    worst = 0.0
    where = None
    for k, (g, r) in enumerate(zip(gs, rs)):
        for c in range(dim + 2):
            e = np.abs(g[c] - r[c]).max() / sc[c]
            if not np.isfinite(e):
                e = np.inf
            if e > worst:
                worst, where = e, (k, c, np.unravel_index(np.abs(g[c] - r[c]).argmax(), g[c].shape))
    return worst, where


def fire_sets_agree(th_gpu, th_ref, tol=1e-9):
    """Faces where a limiter fired (theta < 1) must agree, except at faces where
    theta is within tol of 1 in either code (roundoff-tied decisions). Returns
    (ok, number of mismatching faces, list of tied faces)."""
    fg = th_gpu < 1.0
    fr = th_ref < 1.0
    tied = np.where((np.abs(th_gpu - 1.0) <= tol) | (np.abs(th_ref - 1.0) <= tol))[0]
    mism = np.where(fg != fr)[0]
    bad = np.setdiff1d(mism, tied)
    return len(bad) == 0, len(bad), tied.tolist()
