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


PARITY_TOL = 1e-11      # the FP64 path against the oracle
PARITY_CAP = 1e-10      # the widest bar a roundoff-amplifying problem may take


def parity_bar(p, u0, uo, steps, case=""):
    """The FP64 parity bar of one case: 1e-11, unless the problem itself amplifies a 1-ulp input
    perturbation beyond that (colliding shocks at P3 amplify roundoff about 1e4 in 100 steps, so no
    implementation with a different rounding order can stay within 1e-11 there); then 30x the
    oracle's own measured sensitivity, capped at PARITY_CAP. Prints the bar used (pytest -s)."""
    rng = np.random.default_rng(1)
    up = u0 * (1.0 + 1e-16 * rng.standard_normal(u0.shape))
    ub, _, _ = O.advance(p, up, 0.0, float("inf"), steps)
    sens = rel_l1(p, ub, uo)
    bar = max(PARITY_TOL, 30.0 * sens)
    print("parity bar [%s]: %.3e (oracle 1-ulp sensitivity %.3e)%s"
          % (case, bar, sens, " WIDENED" if bar > PARITY_TOL else ""))
    assert bar <= PARITY_CAP, "case %s amplifies roundoff beyond the cap: %.3e" % (case, bar)
    return bar


def pair(dim=1, nx=16, ny=1, x0=0.0, x1=1.0, y0=0.0, y1=1.0, k=2, eq="burgers", bc="periodic",
         basis="Q", filt=1, cfl=0.1, adv=(1.0, 0.5), precision=N.PREC_FP64, tile_rows=0,
         filter_kind=N.FILTER_JUMP):
    """(oracle Problem, GPU Solver) for the same configuration."""
    b = BC[bc]
    p = O.Problem(dim=dim, nx=nx, ny=ny, x0=x0, x1=x1, y0=y0, y1=y1, bc=(b,) * 4, k=k,
                  basis=O.BASIS_Q if basis == "Q" else O.BASIS_P, eq=EQ[eq][0], filter=filt, cfl=cfl,
                  adv=adv, filter_kind=filter_kind)
    s = N.Solver(dim=dim, nx=nx, ny=ny, x0=x0, x1=x1, y0=y0, y1=y1, bc=(b,) * 4, k=k, eq=EQ[eq][1],
                 filter=filt, cfl=cfl, adv=adv, basis=N.BASIS_Q if basis == "Q" else N.BASIS_P,
                 precision=precision, tile_rows=tile_rows, filter_kind=filter_kind)
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


def l1_vs_finer(pc, uc, pf, uf, var=0):
    """L1 norm over the domain of (coarse solution - finer reference) for variable `var`, both 2D
    Q^k on the same domain with pf.nx = r pc.nx, pf.ny = r pc.ny: integrated cell by cell of the
    finer mesh at its (k+3)^2 Gauss points, the coarse polynomial evaluated there."""
    r = pf.nx // pc.nx
    assert pf.nx == r * pc.nx and pf.ny == r * pc.ny and pc.dim == pf.dim == 2
    kc, kf = pc.k, pf.k
    nq = max(kc, kf) + 3
    xg, wg = npleg.leggauss(nq)

    def vander(k, pts_x, pts_y):
        V1x = np.stack([npleg.legval(pts_x, np.eye(k + 1)[l]) for l in range(k + 1)])
        V1y = np.stack([npleg.legval(pts_y, np.eye(k + 1)[l]) for l in range(k + 1)])
        rows = []
        for q in range(k + 1):
            for p_ in range(k + 1):
                rows.append(np.outer(V1y[q], V1x[p_]).ravel())     # points ordered (y, x)
        return np.stack(rows)                                        # [mode, point]

    W = np.outer(wg, wg).ravel() * (pf.hx * pf.hy / 4.0)
    Vf = vander(kf, xg, xg)
    UF = uf[var].reshape(vander(kf, xg, xg).shape[0], pf.ny, pf.nx)
    UC = uc[var].reshape(-1, pc.ny, pc.nx)
    total = 0.0
    for b in range(r):
        for a in range(r):
            Vc = vander(kc, (2 * a + 1 + xg) / r - 1.0, (2 * b + 1 + xg) / r - 1.0)
            fine = np.einsum("mg,mji->gji", Vf, UF[:, b::r, a::r])
            coarse = np.einsum("mg,mji->gji", Vc, UC)
            total += (W[:, None, None] * np.abs(coarse - fine)).sum()
    return total
