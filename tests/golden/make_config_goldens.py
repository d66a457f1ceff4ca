"""Writes the stored oracle results of the two long workloads the GPU tests
compare with at their full step counts.  It calls only the FP64 oracle
(``oracle/``) and the seeded input recipes (``paper_1112_5547_gb300.inputs``,
which hold no arithmetic of the method); nothing here touches the CUDA path.

  laplace_batch_256.json   D2Q9 Laplace batch: drops of radius R in
                           {8, 12, 16, 20, 24, 28, 32, 40} on 256^2 (seeds 1..8)
                           and a flat interface (slab of half-width 64) on
                           256 x 64 (seed 9), tau = 1, G rho_tot = 2.4,
                           20000 steps each (Sec. 4.1 Laplace test).
  drop3d_128_5000.json     D3Q19 drop R = 32 on 128^3 (seed 2), tau = 1,
                           G rho_tot = 2.4, 5000 steps (the static drop of
                           Sec. 4.1 in three dimensions).

Each file holds the observables of ``observables`` (mass-equivalent radius,
Laplace pressure jump P_in - P_out, peak speed max|u_phys|), the masses of
each species before and after, lines of the fields through the drop centre
and, for the 3D drop, rho_A on every 8th node.  Run from the repository root:

    python tests/golden/make_config_goldens.py [laplace|drop3d|all]

The oracle needs about 20 (laplace) and 40 (drop3d) minutes on 8 cores.
"""
import json
import os
import sys
import time

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

from paper_1112_5547_gb300 import inputs  # noqa: E402

G0 = 2.4 / 1.04  # G (rho_hi + rho_lo) = 2.4 with rho 1.0 / 0.04
LAPLACE_RADII = (8, 12, 16, 20, 24, 28, 32, 40)
LAPLACE_STEPS = 20000
DROP3D_L, DROP3D_STEPS = 128, 5000


def observables(rhoA, p, u, R0):
    """(R, dP, umax) of a drop of nominal radius R0 centred at the box centre.

    R: mass-equivalent radius, the volume V = sum(rho_A - rho_out)/(rho_in - rho_out)
    taken as a disc (2D) or ball (3D), with rho_in the mean over r < R0/4 and
    rho_out the mean over r > R0 + 8 (periodic minimum-image distance r).
    dP: mean bulk pressure over r < R/4 minus the mean over r > R + 8 (Sec. 4.1:
    dP = sigma / R in 2D, 2 sigma / R in 3D).  umax: max |u_phys|."""
    shape = rhoA.shape
    r = inputs.radial_distance(shape, tuple(n / 2.0 for n in reversed(shape)))
    rin = rhoA[r < R0 / 4].mean()
    rout = rhoA[r > R0 + 8].mean()
    V = (rhoA - rout).sum() / (rin - rout)
    R = np.sqrt(V / np.pi) if rhoA.ndim == 2 else (3 * V / (4 * np.pi)) ** (1.0 / 3.0)
    dP = p[r < R / 4].mean() - p[r > R + 8].mean()
    return float(R), float(dP), float(np.sqrt((u ** 2).sum(-1)).max())


def laplace_fit(R, dP):
    """Least-squares dP = sigma / R + c0 in FP64; returns (sigma, c0, r2)."""
    R, dP = np.asarray(R, float), np.asarray(dP, float)
    A = np.vstack([1 / R, np.ones_like(R)]).T
    (sigma, c0), _, _, _ = np.linalg.lstsq(A, dP, rcond=None)
    pred = A @ np.array([sigma, c0])
    r2 = 1 - ((dP - pred) ** 2).sum() / ((dP - dP.mean()) ** 2).sum()
    return float(sigma), float(c0), float(r2)


def slab_jump(p):
    """Bulk pressure inside the slab (x in [96, 160)) minus outside (x < 32 or x >= 224)."""
    return float(p[:, 96:160].mean() - np.concatenate([p[:, :32], p[:, 224:]], axis=1).mean())


def _list(a):
    """Field values rounded to 13 significant digits (far below every tolerance)."""
    return [float("%.13g" % v) for v in np.asarray(a, dtype=np.float64).ravel()]


def laplace_cases():
    """(name, shape, fields, R0) of the D2Q9 Laplace batch."""
    out = [("drop_R%d" % R, (256, 256), inputs.drop((256, 256), R, seed=1 + k), R)
           for k, R in enumerate(LAPLACE_RADII)]
    out.append(("slab", (64, 256), inputs.slab((64, 256), 64, seed=9), None))
    return out


def drop3d_fields():
    L = DROP3D_L
    return inputs.drop((L, L, L), L / 4, seed=2)


def make_laplace(path):
    import oracle
    rec = {"workload": "D2Q9 Laplace batch, tau 1, G rho_tot 2.4, FP64 oracle",
           "steps": LAPLACE_STEPS, "G": G0, "tau": 1.0, "cases": {}}
    R_eq, dPs = [], []
    for name, shape, f, R0 in laplace_cases():
        t0 = time.time()
        o = oracle.OracleSC(0, shape, 1.0, 1.0, G0).init(*f)
        a0, b0, _, _ = o.moments()
        o.step(LAPLACE_STEPS)
        a, b, u, p = o.moments()
        c = {"shape": list(shape), "mass_A0": float(a0.sum()), "mass_B0": float(b0.sum()),
             "mass_A": float(a.sum()), "mass_B": float(b.sum())}
        ny, nx = shape
        if R0 is not None:
            R, dP, umax = observables(a, p, u, R0)
            c.update(R0=R0, R=R, dP=dP, umax=umax,
                     row_rho_A=_list(a[ny // 2]), col_rho_A=_list(a[:, nx // 2]), row_p=_list(p[ny // 2]))
            R_eq.append(R)
            dPs.append(dP)
        else:
            c.update(dP_flat=slab_jump(p), umax=float(np.sqrt((u ** 2).sum(-1)).max()),
                     row_rho_A=_list(a[ny // 2]), row_p=_list(p[ny // 2]))
        rec["cases"][name] = c
        print("%-10s %.0f s" % (name, time.time() - t0), flush=True)
    sigma, c0, r2 = laplace_fit(R_eq, dPs)
    rec["fit"] = {"sigma": sigma, "c0": c0, "r2": r2}
    with open(path, "w") as fh:
        json.dump(rec, fh)


def make_drop3d(path):
    import oracle
    L = DROP3D_L
    t0 = time.time()
    f = drop3d_fields()
    o = oracle.OracleSC(1, (L, L, L), 1.0, 1.0, G0).init(*f)
    a0, b0, _, _ = o.moments()
    o.step(DROP3D_STEPS)
    a, b, u, p = o.moments()
    R, dP, umax = observables(a, p, u, L / 4)
    c = L // 2
    rec = {"workload": "D3Q19 drop R = L/4 on 128^3, tau 1, G rho_tot 2.4, FP64 oracle",
           "steps": DROP3D_STEPS, "G": G0, "tau": 1.0, "shape": [L, L, L], "R0": L / 4,
           "R": R, "dP": dP, "umax": umax,
           "mass_A0": float(a0.sum()), "mass_B0": float(b0.sum()), "mass_A": float(a.sum()), "mass_B": float(b.sum()),
           "line_x_rho_A": _list(a[c, c, :]), "line_y_rho_A": _list(a[c, :, c]), "line_z_rho_A": _list(a[:, c, c]),
           "line_x_rho_B": _list(b[c, c, :]), "line_x_p": _list(p[c, c, :]),
           "sub8_offset": 4, "sub8_rho_A": _list(a[4::8, 4::8, 4::8])}
    with open(path, "w") as fh:
        json.dump(rec, fh)
    print("drop3d %.0f s" % (time.time() - t0), flush=True)


if __name__ == "__main__":
    which = sys.argv[1] if len(sys.argv) > 1 else "all"
    if which in ("laplace", "all"):
        make_laplace(os.path.join(HERE, "laplace_batch_256.json"))
    if which in ("drop3d", "all"):
        make_drop3d(os.path.join(HERE, "drop3d_128_5000.json"))
