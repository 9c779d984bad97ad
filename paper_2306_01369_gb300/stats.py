"""Statistics of a collapsed pile: repose angle and centre of mass (the paper prints no
repose measurement; this is the reading used here).  Used by the long-run statistical
parity test and reported by the benchmark."""
import numpy as np


def pile_statistics(x, m, r_max, centre=(0.0, 0.0)):
    """Pile angle and centre of mass of a collapsed column (the paper reports no
    repose measurement; this is the reading used here).

    Radial bins of width 2 r_max about the initial column axis; the surface height of a
    bin is the 95th percentile of its particles' z (bins with >= 5 particles); a
    least-squares line through the bins whose height lies in [0.2, 0.8] of the tallest
    bin gives the slope, and the angle is atan(-slope) in degrees.  The centre of mass
    is mass-weighted."""
    x = np.asarray(x, np.float64)
    m = np.asarray(m, np.float64)
    rad = np.hypot(x[:, 0] - centre[0], x[:, 1] - centre[1])
    w = 2.0 * r_max
    b = (rad / w).astype(np.int64)
    rs, hs = [], []
    for k in range(int(b.max()) + 1):
        sel = b == k
        if sel.sum() >= 5:
            rs.append((k + 0.5) * w)
            hs.append(np.percentile(x[sel, 2], 95))
    rs, hs = np.array(rs), np.array(hs)
    hmax = hs.max()
    use = (hs >= 0.2 * hmax) & (hs <= 0.8 * hmax)
    slope = np.polyfit(rs[use], hs[use], 1)[0] if use.sum() >= 2 else float("nan")
    com = (m[:, None] * x).sum(0) / m.sum()
    return float(np.degrees(np.arctan(-slope))), com, int(use.sum())
