"""Oracle structured adaptive mesh refinement (AMR) of the step.

TEST INFRASTRUCTURE ONLY (plain PyTorch CPU float64).  Only tests/ and the
bench's CPU baseline may import it.

Cites arXiv 2009.14555:
  * Section 3 (the AMR platform paragraph): refined grids derived recursively
    from coarser ones by a flagging criterion, a hierarchy of embedded
    levels; on level l all mesh widths and the time step are r_l = 2 times
    finer than on level l - 1; the single-grid update is applied to every
    patch of a level (the structured AMR of Berger and Colella: subcycling,
    average-down of the fine solution, refluxing at coarse-fine faces);
  * Section 4.2: difference-based flagging - a cell is tagged when the
    fractional change of a refinement variable to a neighbour exceeds a
    threshold; variables phi_l, phi_l rho_l, u_i and p.

Readings (the paper leaves these to its platform):
  * Blocks.  Level l + 1 refines whole blocks of B x B cells of level l
    (B cells in 1D); a refined block holds 2B x 2B cells of level l + 1.
  * Tags.  A cell is tagged when, against a face neighbour, |a - b| /
    max(|a|, |b|, floor) > eps for a = phi1, phi_l rho_l (l = 1, 2), p and the
    velocity components (floors: 1 for phi1, `u_floor` for velocities, 0
    otherwise); tags are dilated by `buffer` cells; a block is refined when it
    holds a dilated tag and (level l >= 1) its 3^d neighbouring blocks are all
    refined at level l or outside the domain (proper nesting: the ghost
    cells of level l + 1 and the interpolation stencil lie in level l).
  * Ghost cells of level l >= 1 that level l does not own: conservative
    linear interpolation of level l - 1 (per conservative component, slopes
    minmod(q_{i+1} - q_i, q_i - q_{i-1}) along each axis, children at
    -1/4 and +1/4 of the parent width), in time linear between the level
    l - 1 states at the start and the end of its step, at the time of each
    Runge-Kutta stage input (t, t + dt, t + dt / 2).  Domain boundaries keep
    their conditions (applied to the whole level).
  * Time step.  dt_0 = min over levels of 2^l dt_l, dt_l the CFL step of the
    cells level l owns, at the start of each level-0 step; level l then
    takes 2^l steps of dt_0 / 2^l.
  * After the two steps of level l + 1: average-down (each level l cell
    covered by level l + 1 becomes the mean of its 2^d children, every
    component), then refluxing of the conservative rows (phi_l rho_l, rho u,
    rho E, phi_y rho_y lam) at each face between a level l cell not covered
    by level l + 1 and a covered one: the level l flux through that face
    (Runge-Kutta weights 1/6, 1/6, 2/3 over its stages, times dt) is
    replaced by the time- and area-average of the level l + 1 fluxes through
    the same face.  phi1 and V carry non-conservative terms and are not
    refluxed.
  * Cylindrical geometry (x = r, y = z; Section 3, cylindrical symmetry).
    The single-grid scheme is the planar scheme plus the cell-centre
    geometric source s_g, so the conservative variables are per unit (r, z)
    area, and the hierarchy keeps the planar forms above: interpolation,
    average-down and refluxing of those variables (the flux registers hold
    the planar face fluxes); each level adds s_g at its own cell-centre
    radii r = x0 + (i + 1/2) dx_l in every stage.
  * The single-stage MUSCL-Hancock update (oracle/hancock.py; planar) in
    place of SSP-RK3: the ghost cells of level l >= 1 take the coarser
    level's interpolation at the start of each of its steps, and the
    registers hold the corrector's face fluxes times dt (weight 1).
  * Regridding every `regrid_every` level-0 steps, level by level from the
    coarsest: the cells level l does not own first take the interpolation of
    the (current) level l - 1, then level l is tagged; cells that stay
    refined keep their values, new ones take the interpolation of the
    (current) coarser level.

Representation: every level holds a dense array of the whole domain at its
resolution and a mask of the cells it owns; cells it does not own hold the
interpolation of the coarser level and are refilled before every stage.
"""
from __future__ import annotations

import torch

from .closures import cons_to_prim, hencky_dev, mixture_props, phases
from .hancock import hancock_operator_padded
from .scheme import (NG, BC_PERIODIC, F64, _axpy, cfl_rate, fill_ghosts, operator_padded, plastic_update,
                     reaction_update, with_geometric_source)

CONSERVED = ("ar1", "ar2", "mom", "E", "arl")
RK3 = ((0.0, 1.0, 0.0, 1.0 / 6.0), (0.75, 0.25, 1.0, 1.0 / 6.0), (1.0 / 3.0, 2.0 / 3.0, 0.5, 2.0 / 3.0))
# per stage: (a, b, time of the stage input as a fraction of dt, weight of its fluxes in the step)


def _trail(t):
    return (1,) * (t.dim() - 2)


def _minmod(a, b):
    return torch.where(a * b > 0, torch.sign(a) * torch.minimum(a.abs(), b.abs()), torch.zeros_like(a))


def interp_fine(qc, grid_c):
    """Conservative linear interpolation of a dense level to the next finer
    one (ratio 2 in every dimension of grid_c["dim"])."""
    dim = grid_c["dim"]
    g = fill_ghosts(qc, grid_c)
    out = {}
    for k, t in qc.items():
        ny, nx = t.shape[:2]
        gx = g[k] if dim == 1 else g[k][NG:NG + ny]
        c = gx[:, NG:NG + nx]
        sx = _minmod(gx[:, NG + 1:NG + nx + 1] - c, c - gx[:, NG - 1:NG + nx - 1])
        f = torch.repeat_interleave(c, 2, dim=1)
        off = torch.tensor([-0.25, 0.25], dtype=F64).repeat(nx).reshape((1, 2 * nx) + _trail(t))
        f = f + torch.repeat_interleave(sx, 2, dim=1) * off
        if dim == 2:
            gy = g[k][:, NG:NG + nx]
            sy = _minmod(gy[NG + 1:NG + ny + 1] - c, c - gy[NG - 1:NG + ny - 1])
            f = torch.repeat_interleave(f, 2, dim=0)
            offy = torch.tensor([-0.25, 0.25], dtype=F64).repeat(ny).reshape((2 * ny, 1) + _trail(t))
            f = f + torch.repeat_interleave(torch.repeat_interleave(sy, 2, dim=1), 2, dim=0) * offy
        out[k] = f
    return out


def average_down(qf, dim):
    """Mean of the 2^d children of every coarse cell."""
    out = {}
    for k, t in qf.items():
        s = t[:, 0::2] + t[:, 1::2]
        if dim == 2:
            s = s[0::2] + s[1::2]
            out[k] = s / 4.0
        else:
            out[k] = s / 2.0
    return out


def tags(q, mats, dim, eps, u_floor=1.0):
    """Cells whose fractional change of phi1, phi_l rho_l, p or a velocity
    component to a face neighbour exceeds eps (Section 4.2)."""
    w = cons_to_prim(q, mats)
    fields = [(q["phi1"], 1.0), (q["ar1"], 0.0), (q["ar2"], 0.0), (w["p"], 0.0),
              (w["u"][..., 0], u_floor)]
    if dim == 2:
        fields.append((w["u"][..., 1], u_floor))
    tag = torch.zeros(q["phi1"].shape, dtype=torch.bool)
    for a, floor in fields:
        axes = [1] if dim == 1 else [0, 1]
        for ax in axes:
            a0 = a.narrow(ax, 0, a.shape[ax] - 1)
            a1 = a.narrow(ax, 1, a.shape[ax] - 1)
            den = torch.maximum(torch.maximum(a0.abs(), a1.abs()), torch.full_like(a0, floor))
            big = (a1 - a0).abs() > eps * den
            big = big & (den > 0)
            z = torch.zeros_like(tag.narrow(ax, 0, 1))
            tag |= torch.cat([big, z], ax) | torch.cat([z, big], ax)
    return tag


def _dilate(t, n, dim):
    out = t.clone()
    for _ in range(n):
        o = out.clone()
        o[:, 1:] |= out[:, :-1]
        o[:, :-1] |= out[:, 1:]
        if dim == 2:
            o[1:] |= out[:-1]
            o[:-1] |= out[1:]
        out = o
    return out


def _block_any(mask, B, dim):
    ny, nx = mask.shape
    if dim == 1:
        return mask.reshape(1, nx // B, B).any(-1)
    return mask.reshape(ny // B, B, nx // B, B).any(-1).any(1)


def _block_all(mask, B, dim):
    ny, nx = mask.shape
    if dim == 1:
        return mask.reshape(1, nx // B, B).all(-1)
    return mask.reshape(ny // B, B, nx // B, B).all(-1).all(1)


def _expand(blocks, B, dim):
    """Cell mask of the next finer level from a block mask of this level."""
    f = torch.repeat_interleave(blocks, 2 * B, dim=1)
    if dim == 2:
        f = torch.repeat_interleave(f, 2 * B, dim=0)
    return f


class Hierarchy:
    """Levels 0 .. max_level - 1 over one rectangular domain (one patch at
    level 0, boundary conditions grid0["bc"])."""

    def __init__(self, q0, grid0, mats, opts, max_level=2, block=8, eps=0.1, buffer=2,
                 u_floor=1.0, regrid_every=4, extra_tags=None):
        assert opts.get("scheme", "rk3") in ("rk3", "hancock")
        assert grid0.get("geometry", "planar") == "planar" or (
            grid0["geometry"] == "cyl" and opts.get("scheme", "rk3") == "rk3")
        self.extra_tags = extra_tags  # optional (level, grid) -> bool cell mask added to the tags
        self.dim = grid0["dim"]
        self.mats = mats
        self.opts = opts
        self.B = block
        self.eps, self.buffer, self.u_floor = eps, buffer, u_floor
        self.regrid_every = regrid_every
        self.max_level = max_level
        ny, nx = q0["phi1"].shape
        assert nx % block == 0 and (self.dim == 1 or ny % block == 0)
        self.grids = []
        for l in range(max_level):
            g = dict(grid0)
            g["dx"] = grid0["dx"] / 2 ** l
            g["dy"] = grid0["dy"] / 2 ** l if self.dim == 2 else grid0["dy"]
            self.grids.append(g)
        self.q = [q0]
        self.active = [torch.ones((ny, nx), dtype=torch.bool)]
        self.steps = 0
        self.regrid()

    # ---- hierarchy ---------------------------------------------------------
    def _new_blocks(self, l):
        """Block mask (blocks of B cells of level l) of level l + 1."""
        t = tags(self.q[l], self.mats, self.dim, self.eps, self.u_floor)
        if self.extra_tags is not None:
            t = t | self.extra_tags(l, self.grids[l], t.shape)
        t = t & self.active[l]
        t = _dilate(t, self.buffer, self.dim) & self.active[l]
        want = _block_any(t, self.B, self.dim)
        if l >= 1:
            ok = _block_all(self.active[l], self.B, self.dim)
            # every neighbouring block refined at level l (outside the domain counts)
            pad = torch.nn.functional.pad(ok[None, None].to(F64), (1, 1, 1, 1), value=1.0)[0, 0] > 0.5
            if self.dim == 1:
                nb = pad[1:2, :-2] & pad[1:2, 1:-1] & pad[1:2, 2:]
            else:
                nb = torch.ones_like(ok)
                for dj in range(3):
                    for di in range(3):
                        nb = nb & pad[dj:dj + ok.shape[0], di:di + ok.shape[1]]
            want = want & nb
        return want

    def regrid(self):
        """Rebuild levels 1 .. max_level - 1 from the data of the coarser ones."""
        for l in range(self.max_level - 1):
            if l >= 1:  # cells level l does not own: the interpolation of the (current) level l - 1
                f = interp_fine(self.q[l - 1], self.grids[l - 1])
                a = self.active[l]
                self.q[l] = {k: torch.where(a.reshape(a.shape + _trail(v)), v, f[k]) for k, v in self.q[l].items()}
            blocks = self._new_blocks(l)
            act = _expand(blocks, self.B, self.dim)
            fine = interp_fine(self.q[l], self.grids[l])
            if l + 1 < len(self.q):
                keep = act & self.active[l + 1]
                old = self.q[l + 1]
                fine = {k: torch.where(keep.reshape(keep.shape + _trail(v)), old[k], v) for k, v in fine.items()}
                self.q[l + 1] = fine
                self.active[l + 1] = act
            else:
                self.q.append(fine)
                self.active.append(act)
            if not bool(act.any()):
                del self.q[l + 1:]
                del self.active[l + 1:]
                break

    def n_levels(self):
        return len(self.q)

    # ---- time step ---------------------------------------------------------
    def dt0(self):
        dt = None
        for l in range(self.n_levels()):
            r = cfl_rate(self.q[l], self.grids[l], self.mats)
            r = float(r[self.active[l]].max())
            d = self.opts["cfl"] / r * 2 ** l
            dt = d if dt is None else min(dt, d)
        return dt

    def _filled(self, l, qs, theta):
        """Stage input qs of level l with the cells it does not own taken from
        level l - 1 at fraction theta of that level's step."""
        if l == 0:
            return qs
        qc = {k: (1.0 - theta) * self.q_old[l - 1][k] + theta * self.q[l - 1][k] for k in qs}
        f = interp_fine(qc, self.grids[l - 1])
        a = self.active[l]
        return {k: torch.where(a.reshape(a.shape + _trail(v)), v, f[k]) for k, v in qs.items()}

    def _level_step(self, l, dt, t0_frac, frac_len):
        """One SSP-RK3 (or MUSCL-Hancock) step of level l plus sources;
        returns the stage-weighted face fluxes (conservative rows) times dt.
        t0_frac, frac_len: start and length of the step as fractions of the
        step of level l - 1 (for the time interpolation)."""
        g = self.grids[l]
        opts = self.opts
        qn = self.q[l]
        x = qn
        reg = None
        if opts.get("scheme", "rk3") == "hancock":
            # one stage: ghost cells at the start of the step, fluxes of weight 1
            xs = self._filled(l, qn, t0_frac)
            D, faces = hancock_operator_padded(xs, fill_ghosts(xs, g), g, self.mats, opts.get("thinc", False), dt,
                                               opts.get("limiter", "minmod"))
            reg = [{k: dt * F[k] for k in F if k in CONSERVED} for F, _, _, _ in faces]
            x = _axpy(1.0, xs, -dt, D)
        else:
            for a, b, ts, w in RK3:
                xs = self._filled(l, x, t0_frac + ts * frac_len)
                D, faces = operator_padded(xs, fill_ghosts(xs, g), g, self.mats, opts.get("thinc", False),
                                           opts.get("limiter", "minmod"))
                D = with_geometric_source(D, xs, g, self.mats)
                Fw = [{k: w * dt * F[k] for k in F if k in CONSERVED} for F, _, _, _ in faces]
                reg = Fw if reg is None else [{k: r[k] + f[k] for k in r} for r, f in zip(reg, Fw)]
                y = _axpy(1.0, xs, -dt, D)
                x = y if a == 0.0 else _axpy(a, self._filled(l, qn, t0_frac), b, y)
        x = plastic_update(x, self.mats, dt)
        if any(m["reactive"] for m in self.mats):
            x = reaction_update(x, self.mats, dt)
        self.q[l] = x
        return reg

    def _advance(self, l, dt, t0_frac=0.0, frac_len=1.0):
        if l + 1 < self.n_levels():
            self.q_old[l] = self.q[l]
        reg = self._level_step(l, dt, t0_frac, frac_len)
        if l + 1 < self.n_levels():
            freg = None
            for k in range(2):
                r = self._advance(l + 1, dt / 2, k * 0.5, 0.5)
                freg = r if freg is None else [{c: a[c] + b[c] for c in a} for a, b in zip(freg, r)]
            self._sync_down(l, reg, freg)
        return reg

    def _sync_down(self, l, reg_c, reg_f):
        """Average-down of level l + 1 into level l and refluxing of level l."""
        dim = self.dim
        cov = _block_any(self.active[l + 1], 2, dim) if dim == 2 else self.active[l + 1].reshape(1, -1, 2).any(-1)
        avg = average_down(self.q[l + 1], dim)
        qc = {k: torch.where(cov.reshape(cov.shape + _trail(v)), avg[k], v) for k, v in self.q[l].items()}
        g = self.grids[l]
        hs = [g["dx"], g["dy"]]
        for d in range(dim):
            Fc = reg_c[d]
            Ff = reg_f[d]
            # fine fluxes summed over the faces of each coarse face (area average)
            if d == 0:
                Fa = {k: v[:, 0::2] for k, v in Ff.items()}  # coarse face i <- fine face 2i
                if dim == 2:
                    Fa = {k: 0.5 * (v[0::2] + v[1::2]) for k, v in Fa.items()}
                inner = cov  # (ny, nx)
                lo = torch.nn.functional.pad(inner.to(F64), (1, 0))[..., :] > 0.5  # cell left of face f
                hi = torch.nn.functional.pad(inner.to(F64), (0, 1)) > 0.5          # cell right of face f
            else:
                Fa = {k: v[0::2] for k, v in Ff.items()}
                Fa = {k: 0.5 * (v[:, 0::2] + v[:, 1::2]) for k, v in Fa.items()}
                lo = torch.nn.functional.pad(cov.to(F64), (0, 0, 1, 0)) > 0.5
                hi = torch.nn.functional.pad(cov.to(F64), (0, 0, 0, 1)) > 0.5
            cf = lo ^ hi  # a coarse-fine face (one side covered, one not)
            per = g["bc"][2 * d] == BC_PERIODIC
            if per:  # the domain-edge faces see the other end of the domain
                if d == 0:
                    e = cov[:, -1] ^ cov[:, 0]
                    cf[:, 0] = e
                    cf[:, -1] = e
                    lo[:, 0] = cov[:, -1]
                    hi[:, -1] = cov[:, 0]
                else:
                    e = cov[-1] ^ cov[0]
                    cf[0] = e
                    cf[-1] = e
                    lo[0] = cov[-1]
                    hi[-1] = cov[0]
            else:
                if d == 0:
                    cf[:, 0] = False
                    cf[:, -1] = False
                else:
                    cf[0] = False
                    cf[-1] = False
            for k in Fc:
                delta = torch.where(cf.reshape(cf.shape + _trail(Fc[k])), Fa[k] - Fc[k], torch.zeros_like(Fc[k]))
                delta = delta / hs[d]
                # cell c left of face f (face f+1 of c): q_c -= delta_f; right of face f: q_c += delta_f
                if d == 0:
                    upd = -delta[:, 1:] + delta[:, :-1]
                else:
                    upd = -delta[1:] + delta[:-1]
                m = ~cov
                qc[k] = qc[k] + torch.where(m.reshape(m.shape + _trail(upd)), upd, torch.zeros_like(upd))
        self.q[l] = qc

    def step(self):
        """One level-0 step (all levels subcycled); regrids every
        regrid_every level-0 steps afterwards.  Returns dt_0."""
        dt = self.dt0()
        self.q_old = [None] * self.n_levels()
        self._advance(0, dt)
        self.steps += 1
        if self.regrid_every and self.steps % self.regrid_every == 0:
            self.regrid()
        return dt

    def composite_totals(self):
        """Sum of each conservative component times the cell volume over the
        cells no finer level covers."""
        tot = {}
        for l in range(self.n_levels()):
            g = self.grids[l]
            vol = g["dx"] * (g["dy"] if self.dim == 2 else 1.0)
            own = self.active[l].clone()
            if l + 1 < self.n_levels():
                cov = _block_any(self.active[l + 1], 2, self.dim) if self.dim == 2 else \
                    self.active[l + 1].reshape(1, -1, 2).any(-1)
                own &= ~cov
            for k, v in self.q[l].items():
                s = (v[own] * vol).sum(0)
                tot[k] = s if k not in tot else tot[k] + s
        return tot
