"""Shared helpers for the GPU parity tests: problem construction and the relative-L1 measure."""
import os

import numpy as np
from numpy.polynomial import legendre as npleg

import oracle as O
from paper_2407_19169_gb300 import _native as N

O.set_threads(os.cpu_count() or 1)

EQ = {"advection": (O.EQ_ADVECTION, N.EQ_ADVECTION), "burgers": (O.EQ_BURGERS, N.EQ_BURGERS),
      "euler": (O.EQ_EULER, N.EQ_EULER)}
BC = {"periodic": O.BC_PERIODIC, "outflow": O.BC_OUTFLOW}


def pair(dim=1, nx=16, ny=1, x0=0.0, x1=1.0, y0=0.0, y1=1.0, k=2, eq="burgers", bc="periodic",
         basis="Q", filt=1, cfl=0.1, adv=(1.0, 0.5), precision=N.PREC_FP64, tile_rows=0):
    """(oracle Problem, GPU Solver) for the same configuration."""
    b = BC[bc]
    p = O.Problem(dim=dim, nx=nx, ny=ny, x0=x0, x1=x1, y0=y0, y1=y1, bc=(b,) * 4, k=k,
                  basis=O.BASIS_Q if basis == "Q" else O.BASIS_P, eq=EQ[eq][0], filter=filt, cfl=cfl,
                  adv=adv)
    s = N.Solver(dim=dim, nx=nx, ny=ny, x0=x0, x1=x1, y0=y0, y1=y1, bc=(b,) * 4, k=k, eq=EQ[eq][1],
                 filter=filt, cfl=cfl, adv=adv, basis=N.BASIS_Q if basis == "Q" else N.BASIS_P,
                 precision=precision, tile_rows=tile_rows)
    return p, s


def rel_l1(p, a, b, nq=None):
    """max over variables of sum_cells sum_q w_q |a - b| / sum_cells sum_q w_q |b|, evaluated at
    nq Gauss points per direction (default k+3)."""
    nq = nq or p.k + 3
    xg, wg = npleg.leggauss(nq)
    nm = p.nmodes
    if p.dim == 1:
        V = np.stack([npleg.legval(xg, np.eye(p.k + 1)[l]) for l in range(nm)])      # [m, q]
        W = wg
    else:
        V1 = np.stack([npleg.legval(xg, np.eye(p.k + 1)[l]) for l in range(p.k + 1)])
        rows = []
        for m in range(nm):
            pp, qq = mode_pq(p, m)
            rows.append(np.outer(V1[pp], V1[qq]).ravel())
        V = np.stack(rows)
        W = np.outer(wg, wg).ravel()
    worst = 0.0
    for v in range(p.nvars):
        da = np.abs(V.T @ (a[v] - b[v]))        # [q, cell]
        db = np.abs(V.T @ b[v])
        num = (W[:, None] * da).sum()
        den = (W[:, None] * db).sum()
        worst = max(worst, num / den if den > 0 else num)
    return worst


def mode_pq(p, m):
    if p.dim == 1:
        return m, 0
    idx = 0
    for q in range(p.k + 1):
        for pp in range(p.k + 1):
            if p.basis == O.BASIS_P and pp + q > p.k:
                continue
            if idx == m:
                return pp, q
            idx += 1
    raise IndexError(m)
