"""Guard-band accounting for FP32 binning gates (test helper, uses the oracle).

A sample copy whose oracle coordinate lies within `band` bin widths of a bin
edge may legitimately land in the neighbouring bin when the trajectory is
integrated in FP32.  These helpers count such (copy, coordinate) events per
orbit from the oracle's own trajectory so that the gates can allow exactly
those moves and nothing else."""
import numpy as np


def guard_events(orc, pot, omega, dt, S, ics, grid, band):
    po = orc.make_pot(pot)
    R = orc.euler_matrix(grid.get("bar_angle", 0.0), grid["incl"], grid.get("pa", 0.0))
    nx, ny, pix = grid["nx"], grid["ny"], grid["pix"]
    x0, y0 = -0.5 * nx * pix, -0.5 * ny * pix
    dR = grid.get("Rmax", 10.0) / grid["nR"]
    dphi = 2 * np.pi / grid["nphi"]
    zmin, zmax = grid.get("zmin", -3.0), grid.get("zmax", 3.0)
    dz = (zmax - zmin) / grid["nz"]
    gh = bool(grid.get("gh"))
    if not gh:
        vmax, nv = grid.get("vmax", 400.0), grid["nv"]
        dv = 2 * vmax / nv
    th = omega * dt * np.arange(1, S + 1)
    c, s = np.cos(th), np.sin(th)
    out = np.zeros(len(ics), dtype=np.int64)
    for i, ic in enumerate(ics):
        tr = orc.trajectory(po, omega, dt, S, ic)[1:]
        xb = c * tr[:, 0] + s * tr[:, 1]; yb = -s * tr[:, 0] + c * tr[:, 1]; zb = tr[:, 2]
        vxb = c * tr[:, 3] + s * tr[:, 4]; vyb = -s * tr[:, 3] + c * tr[:, 4]; vzb = tr[:, 5]
        n = 0
        for sx, sz in [(1, 1), (1, -1), (-1, 1), (-1, -1)]:
            p = np.stack([sx * xb, sx * yb, sz * zb]); v = np.stack([sx * vxb, sx * vyb, sz * vzb])
            X, Y = R[0] @ p, R[1] @ p
            coords = [(X - x0) / pix, (Y - y0) / pix, np.hypot(p[0], p[1]) / dR,
                      (np.arctan2(p[1], p[0]) % (2 * np.pi)) / dphi, (p[2] - zmin) / dz]
            if not gh:
                coords.append(((R[2] @ v) + vmax) / dv)
            for u in coords:
                n += int(np.sum(np.abs(u - np.rint(u)) < band))
        out[i] = n
    return out
