"""Sub-volumes of a problem for cell-by-cell checks of full-size runs: a
box of half-width H around a cell, wrapping periodic x and y, clipped at the
z walls, with outflow sides where it cuts the domain (no test here)."""
import numpy as np

import workloads as W


def sub_problem(pr, c, H):
    """Sub-box of pr centred on cell c = (i, j, k): x, y wrap (periodic domain),
    z clipped at the walls; returns (problem, index arrays of the sub-box)."""
    nz = pr.n[2]
    ix = np.arange(c[0] - H, c[0] + H + 1) % pr.n[0]
    iy = np.arange(c[1] - H, c[1] + H + 1) % pr.n[1]
    z0, z1 = max(0, c[2] - H), min(nz, c[2] + H + 1)
    iz = np.arange(z0, z1)
    q = pr.copy()
    nx, ny, nzs = ix.size, iy.size, iz.size
    q.n = (nx, ny, nzs)
    dx = [(pr.hi[d] - pr.lo[d]) / pr.n[d] for d in range(3)]
    q.lo = (0.0, 0.0, pr.lo[2] + z0 * dx[2])
    q.hi = (nx * dx[0], ny * dx[1], pr.lo[2] + z1 * dx[2])
    q.bc = ((W.OUTFLOW, W.OUTFLOW), (W.OUTFLOW, W.OUTFLOW),
            (W.REFLECT if z0 == 0 else W.OUTFLOW, W.REFLECT if z1 == nz else W.OUTFLOW))
    sel = np.ix_(iz, iy, ix)
    q.cons = np.ascontiguousarray(pr.cons[(slice(None),) + sel])
    q.bx = np.ascontiguousarray(pr.bx[np.ix_(iz, iy, np.append(ix, (ix[-1] + 1) % (pr.n[0] + 1)))])
    q.by = np.ascontiguousarray(pr.by[np.ix_(iz, np.append(iy, (iy[-1] + 1) % (pr.n[1] + 1)), ix)])
    q.bz = np.ascontiguousarray(pr.bz[np.ix_(np.arange(z0, z1 + 1), iy, ix)])
    q.bg = {"rho_c": pr.bg["rho_c"][z0:z1 + 6], "p_c": pr.bg["p_c"][z0:z1 + 6],
            "rho_f": pr.bg["rho_f"][z0:z1 + 7], "p_f": pr.bg["p_f"][z0:z1 + 7]}
    q.heat = None if pr.heat is None else np.ascontiguousarray(pr.heat[z0:z1])
    return q, (ix, iy, iz)
