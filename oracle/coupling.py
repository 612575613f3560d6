"""Fluid-particle coupling of the oracle: boundary conditions, momentum
exchange, missing links and PDF refill.

Test infrastructure only (see ``oracle/__init__.py``).

Paper passages followed (Sec. 2.2):
  * Eq. (2): pull form of the streaming step f_q(x, t+1) = f~_q(x - c_q, t).
  * Eq. (14): CLI moving no-slip condition, falling back to bounce-back
    (delta_q = 1/2) when the cell x - c_q (paper notation) is not fluid.
  * Eq. (15): Galilean-invariant momentum exchange per link; Eqs. (16)-(17):
    per-particle force and torque sums.
  * missing fluid-solid links near other bodies get F_q = 2 w_q c_q.
  * Eq. (18): refill of cells uncovered by a particle.
Readings where the paper is silent or ambiguous:
  * walls sit halfway between cells on the domain faces; a wall link uses
    Eq. (14) with delta = 1/2 and the face velocity as u_b and adds no force.
  * in the bounce-back fallback only the coefficients of Eq. (14) take
    delta = 1/2; x_b and u_b stay at the true surface point.
  * a missing link of particle i is a link x -> s with s a solid cell of i
    and x a cell of another body (another particle, or outside the domain
    behind a wall) whose centre is not inside sphere i.
  * refill: rho_bar is the mean density of the D3Q19 neighbours that are
    fluid before and after the mapping update (rho0 if there is none); the
    derivative along axis b is central when both axis neighbours are such
    cells, one-sided against u_t when only one is, zero otherwise; the
    neighbour velocity is the physical one of its post-collision PDFs.
"""
import numpy as np

from .d3q19 import C, W, OPP, Q, CS2, RHO0
from .lbm import density, velocity_from_post_collision
from .particles import link_fraction, rel_vec, dist2


def _shift(pos, c, dom):
    """Neighbour index pos + c with periodic wrap; outside a wall axis the
    neighbour is the wall of Eq. (14) with delta = 1/2. Returns (idx, out,
    wall_axis)."""
    n = dom.shape
    idx = pos + np.asarray(c, dtype=np.int64)
    out = np.zeros(len(pos), dtype=bool)
    wall_axis = np.full(len(pos), -1, dtype=np.int64)
    for a in range(3):
        if dom.periodic[a]:
            idx[:, a] %= n[a]
        else:
            o = (idx[:, a] < 0) | (idx[:, a] >= n[a])
            wall_axis = np.where(o & (wall_axis < 0), a, wall_axis)
            out |= o
    return idx, out, wall_axis


def _at(arr, idx):
    """arr[..., z, y, x] gathered at integer positions idx (K, 3) = (x, y, z)
    (indexing helper)."""
    return arr[..., idx[:, 2], idx[:, 1], idx[:, 0]]


def stream_and_couple(ft, dom, owner, X, U, Om, R):
    """Boundary conditions, pull streaming and momentum exchange (Alg. 1,
    first two lines; Eqs. (2), (14)-(17)).

    ft: post-collision PDFs f~(t) (19, nz, ny, nx), valid in fluid cells.
    owner: (nz, ny, nx) particle index of solid cells, -1 for fluid.
    Returns f(t+1) before collision (valid in fluid cells) and the per
    particle force and torque sums of Eqs. (16)-(17).
    """
    nx, ny, nz = dom.shape
    npart = len(R)
    F = np.zeros((npart, 3))
    T = np.zeros((npart, 3))
    fluid = owner < 0
    Z, Y, Xc = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing='ij')
    grid_pos = (Xc, Y, Z)
    f = np.zeros_like(ft)
    for q in range(Q):
        c = C[q]
        p = OPP[q]
        cp = C[p].astype(np.float64)
        # Eq. (2) in pull form: f_q(x, t+1) = f~_q(x - c_q, t), periodic wrap
        val = np.roll(ft[q], shift=(c[2], c[1], c[0]), axis=(0, 1, 2))
        # upstream cell x - c_q outside the box on a wall axis -> wall link
        out = np.zeros(owner.shape, dtype=bool)
        for a in (2, 1, 0):
            if dom.periodic[a] or c[a] == 0:
                continue
            up = grid_pos[a] - c[a]
            for side, o in ((0, up < 0), (1, up >= dom.shape[a])):
                o = o & ~out
                if o.any():
                    uw = dom.wall_vel[side][a]
                    # Eq. (14) with delta = 1/2: halfway bounce-back with wall velocity
                    val[o] = ft[p][o] - 6.0 * W[p] * RHO0 * (uw @ cp)
                    out |= o
        up_owner = np.roll(owner, shift=(c[2], c[1], c[0]), axis=(0, 1, 2))
        links = fluid & ~out & (up_owner >= 0)
        iz, iy, ix = np.nonzero(links)
        if len(iz):
            pos = np.stack([ix, iy, iz], axis=-1).astype(np.int64)
            i = up_owner[iz, iy, ix]
            xc = pos + 0.5
            delta = link_fraction(xc, cp, X[i], R[i], dom)
            down, dout, _ = _shift(pos, c, dom)
            down_fluid = np.zeros(len(pos), dtype=bool)
            down_fluid[~dout] = _at(owner, down[~dout]) < 0
            xb = xc + delta[:, None] * cp
            r = rel_vec(xb, X[i], dom)
            ub = U[i] + np.cross(Om[i], r)
            dbc = np.where(down_fluid, delta, 0.5)
            kappa = (1.0 - 2.0 * dbc) / (1.0 + 2.0 * dbc)
            f_down = np.zeros(len(pos))
            f_down[down_fluid] = _at(ft[p], down[down_fluid])
            f_out = ft[p][iz, iy, ix]           # f~ towards the surface
            f_in = ft[q][iz, iy, ix]            # f~ away from the surface
            v = f_out + kappa * (f_down - f_in) - 12.0 * W[p] / (1.0 + 2.0 * dbc) * RHO0 * (ub @ cp)
            val[iz, iy, ix] = v
            # Eq. (15): F = (c_p - u_b) f~_p(x) - (c_q - u_b) f_q(x, t+1)
            Fl = (cp - ub) * f_out[:, None] - (c.astype(np.float64) - ub) * v[:, None]
            np.add.at(F, i, Fl)
            np.add.at(T, i, np.cross(r, Fl))
        f[q] = np.where(fluid, val, 0.0)
    return f, F, T


def missing_links(dom, owner, X, R):
    """Missing-link correction F_q = 2 w_q c_q of Sec. 2.2 (reading above).

    Returns per-particle force and torque contributions.
    """
    npart = len(R)
    F = np.zeros((npart, 3))
    T = np.zeros((npart, 3))
    iz, iy, ix = np.nonzero(owner >= 0)
    spos = np.stack([ix, iy, iz], axis=-1).astype(np.int64)
    own = owner[iz, iy, ix]
    for q in range(1, Q):
        c = C[q]
        cf = c.astype(np.float64)
        xpos, out, _ = _shift(spos, -c, dom)
        other = np.zeros(len(spos), dtype=bool)
        xo = _at(owner, xpos[~out])
        other[~out] = (xo >= 0) & (xo != own[~out])
        cand = np.nonzero(out | other)[0]
        if not len(cand):
            continue
        i = own[cand]
        # unwrapped virtual cell centre on the far side of the link
        xc = (spos[cand] - c) + 0.5
        d2 = dist2(xc, X[i], dom)
        keep = d2 > R[i] * R[i]
        cand, i, xc = cand[keep], i[keep], xc[keep]
        if not len(cand):
            continue
        delta = link_fraction(xc, cf, X[i], R[i], dom)
        r = rel_vec(xc + delta[:, None] * cf, X[i], dom)
        Fm = np.broadcast_to(2.0 * W[q] * RHO0 * cf, (len(cand), 3))
        np.add.at(F, i, Fm)
        np.add.at(T, i, np.cross(r, Fm))
    return F, T


def refill(ft, dom, owner_old, owner_new, X, U, Om, s_nu, accel):
    """Eq. (18): reconstruct PDFs in cells that went from solid to fluid.

    Modifies ft in place and returns the list of refilled cells (x, y, z).
    """
    new_fluid = (owner_old >= 0) & (owner_new < 0)
    both = (owner_old < 0) & (owner_new < 0)
    rho = density(ft)
    u = velocity_from_post_collision(ft, accel)
    n = dom.shape
    cells = []
    for z, y, x in zip(*np.nonzero(new_fluid)):
        pos = np.array([x, y, z], dtype=np.int64)
        i = owner_old[z, y, x]

        def neighbour(c):
            """Neighbour pos + c if it is fluid before and after the update
            (the cells Eq. (18)'s averages and differences may use), else None."""
            nb = pos + c
            for a in range(3):
                if dom.periodic[a]:
                    nb[a] %= n[a]
                elif nb[a] < 0 or nb[a] >= n[a]:
                    return None
            return nb if both[nb[2], nb[1], nb[0]] else None

        rs = []
        for q in range(1, Q):
            nb = neighbour(C[q])
            if nb is not None:
                rs.append(rho[nb[2], nb[1], nb[0]])
        rho_bar = float(np.mean(rs)) if rs else RHO0
        r = rel_vec((pos + 0.5)[None, :], X[i], dom)[0]
        u_t = U[i] + np.cross(Om[i], r)
        grad = np.zeros((3, 3))          # grad[a, b] = d u_a / d x_b
        for b in range(3):
            e = np.zeros(3, dtype=np.int64)
            e[b] = 1
            up, dn = neighbour(e), neighbour(-e)
            if up is not None and dn is not None:
                grad[:, b] = 0.5 * (u[:, up[2], up[1], up[0]] - u[:, dn[2], dn[1], dn[0]])
            elif up is not None:
                grad[:, b] = u[:, up[2], up[1], up[0]] - u_t
            elif dn is not None:
                grad[:, b] = u_t - u[:, dn[2], dn[1], dn[0]]
        strain = grad + grad.T
        for q in range(Q):
            cq = C[q].astype(np.float64)
            second = 0.0
            for a in range(3):
                for b in range(3):
                    pab = rho_bar * u_t[a] * u_t[b] - rho_bar * CS2 / s_nu * strain[a, b]
                    second += pab * (cq[a] * cq[b] - CS2 * (1.0 if a == b else 0.0))
            ft[q, z, y, x] = W[q] * (rho_bar + rho_bar * (u_t @ cq) / CS2 + second / (2.0 * CS2 * CS2))
        cells.append((int(x), int(y), int(z)))
    return cells
