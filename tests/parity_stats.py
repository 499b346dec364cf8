"""Two-sample statistics for comparing Monte Carlo tallies of the CUDA path
with the oracle's on independent packets (test infrastructure only).

Packets are independent, but the peel-off contributions of one packet are
not (a packet adds to the same camera bins at many scatterings), so the
weighted tallies are compared through batch means: each side is run as B
batches of n packets, and the per-packet mean of every bin is estimated with
the spread of its batch means.
"""
import numpy as np
from scipy import stats


def binomial_sigma(k1, n1, k2, n2):
    """(difference of the two fractions in units of its standard error under
    a common p, that standard error)."""
    p = (k1 + k2) / (n1 + n2)
    se = np.sqrt(max(p * (1 - p), 0.0) * (1.0 / n1 + 1.0 / n2))
    d = k1 / n1 - k2 / n2
    return (0.0 if d == 0 else np.inf) if se == 0 else d / se, se


def merge_counts(a, b, min_count=10):
    """Merge adjacent bins (left to right) until each merged bin holds at
    least min_count entries of a + b; a last short group joins its left
    neighbour.  Returns the merged (a, b)."""
    a, b = np.asarray(a, float), np.asarray(b, float)
    groups, cur = [], []
    tot = 0.0
    for i in range(len(a)):
        cur.append(i)
        tot += a[i] + b[i]
        if tot >= min_count:
            groups.append(cur)
            cur, tot = [], 0.0
    if cur:
        if groups:
            groups[-1] += cur
        else:
            groups.append(cur)
    ma = np.array([a[g].sum() for g in groups])
    mb = np.array([b[g].sum() for g in groups])
    return ma, mb


def two_sample_counts(a, b, min_count=10):
    """Two-sample chi-square test of histograms of counts (a: n_a packets, b:
    n_b packets, unequal totals allowed) after merging sparse bins.  Returns
    (chi2, dof, p)."""
    a, b = merge_counts(a, b, min_count)
    na, nb = a.sum(), b.sum()
    m = (a + b) > 0
    if np.count_nonzero(m) < 2 or na == 0 or nb == 0:
        return 0.0, 0, 1.0
    k1, k2 = np.sqrt(nb / na), np.sqrt(na / nb)
    chi2 = float(np.sum((k1 * a[m] - k2 * b[m]) ** 2 / (a[m] + b[m])))
    dof = int(np.count_nonzero(m) - 1)
    return chi2, dof, float(stats.chi2.sf(chi2, dof))


def merge_weighted(sum_a, sq_a, sum_b, sq_b, min_eff=30.0):
    """Groups of adjacent bins such that both samples have an effective number
    of contributions (sum w)^2 / sum w^2 of at least min_eff in every group
    (bins empty on both sides are dropped).  Returns a list of index lists."""
    groups, cur = [], []
    sa = qa = sb = qb = 0.0
    for i in range(len(sum_a)):
        if sum_a[i] == 0 and sum_b[i] == 0 and not cur:
            continue
        cur.append(i)
        sa, qa, sb, qb = sa + sum_a[i], qa + sq_a[i], sb + sum_b[i], qb + sq_b[i]
        ea = sa * sa / qa if qa > 0 else 0.0
        eb = sb * sb / qb if qb > 0 else 0.0
        if ea >= min_eff and eb >= min_eff:
            groups.append(cur)
            cur, sa, qa, sb, qb = [], 0.0, 0.0, 0.0, 0.0
    if cur and groups:
        groups[-1] += cur
    return groups


def batch_means_test(xa, xb):
    """Welch comparison of per-packet bin means from batches.

    xa: (B_a, k) per-packet means of each batch of sample a, xb: (B_b, k).
    Each bin's Welch t is mapped to a standard normal z through its
    Welch-Satterthwaite t distribution; the sum of z^2 over the bins is
    referred to chi-square with k degrees of freedom.  Returns (z, chi2, p)."""
    xa, xb = np.asarray(xa, float), np.asarray(xb, float)
    Ba, Bb = xa.shape[0], xb.shape[0]
    ma, mb = xa.mean(axis=0), xb.mean(axis=0)
    va, vb = xa.var(axis=0, ddof=1) / Ba, xb.var(axis=0, ddof=1) / Bb
    se = np.sqrt(va + vb)
    ok = se > 0
    t = np.zeros_like(ma)
    t[ok] = (ma[ok] - mb[ok]) / se[ok]
    with np.errstate(divide="ignore", invalid="ignore"):
        nu = (va + vb) ** 2 / (va ** 2 / (Ba - 1) + vb ** 2 / (Bb - 1))
    nu = np.where(np.isfinite(nu), nu, max(Ba, Bb) - 1)
    z = np.zeros_like(t)
    z[ok] = stats.norm.isf(stats.t.sf(t[ok], nu[ok]))
    z = np.clip(z, -40, 40)
    k = int(np.count_nonzero(ok))
    chi2 = float(np.sum(z[ok] ** 2))
    return z[ok], chi2, (float(stats.chi2.sf(chi2, k)) if k else 1.0)


def camera_spectra_test(ga, gb, min_eff=30.0):
    """Compare camera spectra of two batch sets.

    ga, gb: lists of (cam_spec, cam_spec2, n_packets) per batch, cam_spec of
    shape (n_cam, nbins).  Bins are merged per camera so that both samples
    have min_eff effective contributions per group.  Returns per camera
    (n_groups, chi2, p) and the largest relative difference of the pooled
    per-packet means over groups."""
    out = []
    n_cam = ga[0][0].shape[0]
    for c in range(n_cam):
        Sa = sum(b[0][c] for b in ga)
        Qa = sum(b[1][c] for b in ga)
        Sb = sum(b[0][c] for b in gb)
        Qb = sum(b[1][c] for b in gb)
        groups = merge_weighted(Sa, Qa, Sb, Qb, min_eff)
        if len(groups) < 2:
            out.append(dict(groups=len(groups), chi2=0.0, p=1.0, max_rel=0.0))
            continue
        xa = np.array([[b[0][c][g].sum() / b[2] for g in groups] for b in ga])
        xb = np.array([[b[0][c][g].sum() / b[2] for g in groups] for b in gb])
        z, chi2, p = batch_means_test(xa, xb)
        ma, mb = xa.mean(axis=0), xb.mean(axis=0)
        rel = np.abs(ma - mb) / np.maximum(np.abs(mb), 1e-300)
        out.append(dict(groups=len(groups), chi2=chi2, p=p, max_rel=float(rel.max())))
    return out


def block_image(cube, npix, nbins, block_pix):
    """Image cube [v][u][bin] of one camera summed over the spectral bins and
    pooled into block_pix x block_pix pixel blocks -> (npix/block_pix)^2."""
    img = np.asarray(cube).reshape(npix, npix, nbins).sum(axis=2)
    nb = npix // block_pix
    return img.reshape(nb, block_pix, nb, block_pix).sum(axis=(1, 3)).ravel()


def image_blocks_test(xa, xb, min_nonzero=0.75):
    """Compare pooled image blocks of two batch sets: xa (B_a, k), xb (B_b, k)
    per-packet block means.  Blocks that are nonzero in fewer than
    min_nonzero of the batches of either sample are left out (their batch
    means are far from normal).  Returns (blocks used, chi2, p)."""
    xa, xb = np.asarray(xa, float), np.asarray(xb, float)
    use = (np.mean(xa > 0, axis=0) >= min_nonzero) & (np.mean(xb > 0, axis=0) >= min_nonzero)
    if np.count_nonzero(use) < 2:
        return int(np.count_nonzero(use)), 0.0, 1.0
    z, chi2, p = batch_means_test(xa[:, use], xb[:, use])
    return int(np.count_nonzero(use)), chi2, p


def permutation_test(xa, xb, n_perm=20000, seed=12345, chunk=500):
    """Two-sample permutation test of bin means from equal-size batches.

    xa (B_a, k), xb (B_b, k): the per-packet mean of every bin in each batch;
    all batches hold the same number of packets, so under the null hypothesis
    (one distribution) the B_a + B_b batches are exchangeable whatever the
    shape of that distribution (peel-off weights are heavy-tailed).  The
    statistic T = sum_bins (mean_a - mean_b)^2 / s^2, with s^2 the variance of
    the pooled batches (unchanged by relabelling), is compared with its value
    over random relabellings.  Bins with no spread in the pool are skipped.
    Returns (bins used, T, p) with p = (1 + #{T_perm >= T}) / (1 + n_perm)."""
    xa, xb = np.asarray(xa, float), np.asarray(xb, float)
    pool = np.concatenate([xa, xb], axis=0)
    s2 = pool.var(axis=0, ddof=1)
    use = s2 > 0
    if np.count_nonzero(use) == 0:
        return 0, 0.0, 1.0
    pool = pool[:, use] / np.sqrt(s2[use])
    Ba = xa.shape[0]
    n = pool.shape[0]
    tot = pool.sum(axis=0)

    def stat(sa):                      # sa: (..., k) sums over the relabelled sample a
        return np.sum((sa / Ba - (tot - sa) / (n - Ba)) ** 2, axis=-1)
    t_obs = float(stat(pool[:Ba].sum(axis=0)))
    rng = np.random.default_rng(seed)
    ge = 0
    done = 0
    while done < n_perm:
        m = min(chunk, n_perm - done)
        idx = np.argsort(rng.random((m, n)), axis=1)[:, :Ba]
        ge += int(np.count_nonzero(stat(pool[idx].sum(axis=1)) >= t_obs))
        done += m
    return int(np.count_nonzero(use)), t_obs, (1.0 + ge) / (1.0 + n_perm)


def camera_permutation_test(ga, gb, min_eff=30.0, n_perm=20000):
    """Camera spectra of two batch sets of equal batch size: ga, gb lists of
    (cam_spec, cam_spec2, n_packets) per batch.  Bins are merged per camera
    to min_eff effective contributions on each side (as merge_weighted), and
    each camera is a permutation test over the merged bins.  Returns per
    camera (groups, T, p, max_rel) with max_rel the largest relative
    difference of the two per-packet group means."""
    out = []
    n_cam = ga[0][0].shape[0]
    for c in range(n_cam):
        Sa = sum(b[0][c] for b in ga)
        Qa = sum(b[1][c] for b in ga)
        Sb = sum(b[0][c] for b in gb)
        Qb = sum(b[1][c] for b in gb)
        groups = merge_weighted(Sa, Qa, Sb, Qb, min_eff)
        if len(groups) < 1:
            out.append(dict(groups=0, T=0.0, p=1.0, max_rel=0.0))
            continue
        xa = np.array([[b[0][c][g].sum() / b[2] for g in groups] for b in ga])
        xb = np.array([[b[0][c][g].sum() / b[2] for g in groups] for b in gb])
        k, T, p = permutation_test(xa, xb, n_perm)
        ma, mb = xa.mean(axis=0), xb.mean(axis=0)
        rel = np.abs(ma - mb) / np.maximum(np.abs(mb), 1e-300)
        out.append(dict(groups=len(groups), T=T, p=p, max_rel=float(rel.max())))
    return out
