"""Pins of the oracle's boundary update (Algorithm 1 of Sec. 3.1 fills the
ghost layers before the primitives are used; Sec. 4.2 uses walls and
zero-gradient boundaries; the jet's x-low side is an inflow disc).  No GPU.

Each boundary kind is fixed by something other than the oracle's own
mapping: an equivalent problem without that boundary kind (a mirror-extended
periodic domain for a wall, a domain extended by the ghost states the
boundary kind stands for), the conservation a closed box must show, and the
exact Euler flux that a zero-gradient face must carry.
"""
import dataclasses

import numpy as np
import pytest

import oracle
from paper_2304_00140_gb300 import workloads as wl

P_, R_, O_, I_ = wl.BC_PERIODIC, wl.BC_REFLECT, wl.BC_OUTFLOW, wl.BC_INFLOW


def _axis(d):
    """array axis of grid dimension d in the [nv, nz, ny, nx] layout"""
    return 3 - d


def _rel_max(a, b):
    a = a.reshape(a.shape[0], -1)
    b = b.reshape(b.shape[0], -1)
    return (np.abs(a - b).max(axis=1) / np.maximum(np.abs(b).max(axis=1), 1e-300)).max()


def _resize(w, d, n_new, bc_d):
    n = list(w.n)
    hi = list(w.hi)
    bc = [list(b) for b in w.bc]
    hi[d] = w.lo[d] + w.dx[d] * n_new
    n[d] = n_new
    bc[d] = list(bc_d)
    return dataclasses.replace(w, n=n, hi=hi, bc=bc, inflow=None)


WALL_CASES = {
    "2d_x_plain": dict(d=0, kw=dict()),
    "2d_y_iles_csf_3comp": dict(d=1, kw=dict(ncomp=3, iles=1, sigma=5.0)),
    "2d_x_hf": dict(d=0, kw=dict(sigma=5.0, curvature=1)),
    "3d_z_iles_csf": dict(d=2, ndim=3, kw=dict(iles=1, sigma=5.0)),
    "2d_y_capillary_jump": dict(d=1, kw=dict(sigma=5.0, st_model=1)),
}


@pytest.mark.parametrize("name", sorted(WALL_CASES))
def test_reflective_walls_equal_mirror_extended_periodic_domain(name):
    """A box with reflective walls on both sides of dimension d evolves
    exactly like the right half of a periodic box of twice the length whose
    left half holds the mirror image (normal momentum negated): there both
    walls are planes of mirror symmetry.  An off-by-one mirror, a missing or
    misplaced normal-velocity flip, or a wrong second ghost layer breaks the
    equality."""
    c = WALL_CASES[name]
    d, nd = c["d"], c.get("ndim", 2)
    n = (12, 10) if nd == 2 else (8, 7, 8)
    bc = [[P_, P_], [P_, P_], [P_, P_]]
    bc[d] = [R_, R_]
    w = wl.random_state(n=n, ndim=nd, bc=bc, **c["kw"])
    o = oracle.Oracle(w)
    q = o.prim_to_cons(w.primitives())
    ax = _axis(d)
    mirror = np.flip(q, axis=ax).copy()
    mirror[1 + d] *= -1.0
    qe = np.concatenate([mirror, q], axis=ax)
    we = _resize(w, d, 2 * w.n[d], (P_, P_))
    oe = oracle.Oracle(we)
    assert oe.dt(qe, w.cfl) == o.dt(q, w.cfl)
    got, _ = o.step(q, 3, w.cfl)
    ext, _ = oe.step(qe, 3, w.cfl)
    half = np.take(ext, np.arange(w.n[d], 2 * w.n[d]), axis=ax)
    assert _rel_max(got, half) <= 1e-14, _rel_max(got, half)
    assert np.abs(got - q).max() > 0


def test_closed_reflective_box_conserves_mass_energy_and_species():
    """Walls on every side: no mass, energy or species crosses a wall (the
    mirror states give u* = 0 at the wall face, Eq. 3-2), so those totals
    stay constant to rounding over a run (sigma = 0: the CSF source is not in
    divergence form)."""
    w = wl.random_state(n=(20, 18), ncomp=3, bc=[[R_, R_], [R_, R_], [P_, P_]])
    o = oracle.Oracle(w)
    q = o.prim_to_cons(w.primitives())
    t0 = o.totals(q)
    q1, _ = o.step(q, 10, w.cfl)
    t1 = o.totals(q1)
    keep = [0, 1 + w.ndim] + list(range(2 + w.ndim, w.nvar))
    for v in keep:
        assert abs(t1[v] - t0[v]) <= 1e-13 * abs(t0[v]), (v, t0[v], t1[v])
    # the walls do exert a force: momentum is not conserved
    assert np.abs(q1[1:1 + w.ndim] - q[1:1 + w.ndim]).max() > 0


def _euler_flux(o, W, d):
    """exact Euler flux along d of primitive cell states W[nv, ...] through
    the closure (Eq. 2-2 C with rho H = rho E + p)"""
    nd = o.w.ndim
    Wf = W.reshape(W.shape[0], -1)
    F = np.zeros_like(Wf)
    for c in range(Wf.shape[1]):
        u = Wf[:nd, c]
        p, T, Yt = Wf[nd, c], Wf[nd + 1, c], Wf[nd + 2:, c]
        rho, e, _, _ = o.forward(p, T, Yt)
        E = e + 0.5 * (u * u).sum()
        un = u[d]
        F[0, c] = rho * un
        F[1:1 + nd, c] = rho * un * u
        F[1 + d, c] += p
        F[1 + nd, c] = un * (rho * E + p)
        F[2 + nd:, c] = rho * un * Yt
    return F.reshape(W.shape)


@pytest.mark.parametrize("ndim", [1, 2])
def test_outflow_face_carries_the_euler_flux_of_the_edge_cell(ndim):
    """Zero-gradient outflow: the ghost cells copy the edge cell, so at the
    boundary face both reconstructions (Sec. 3.3) return the edge cell's
    state and the all-Mach flux (Eq. 3-1/3-2) reduces to the exact Euler
    flux.  Summed over a stage, every interior face telescopes and the totals
    change by exactly -a dt (F(W_last) - F(W_first)) / dx along x."""
    if ndim == 1:
        w = wl.random_state(n=(40, 1), ndim=2, bc=[[O_, O_], [P_, P_], [P_, P_]])
        w = dataclasses.replace(w, ndim=1, n=[40, 1, 1], hi=[w.hi[0], 1.0, 1.0],
                                bc=[[O_, O_], [P_, P_], [P_, P_]])
    else:
        w = wl.random_state(n=(24, 10), bc=[[O_, O_], [P_, P_], [P_, P_]])
    o = oracle.Oracle(w)
    W = w.primitives()
    # ramps along x so that the two boundary faces carry different fluxes
    ramp = np.linspace(-1.0, 1.0, w.n[0])
    W[0] += 60.0 * ramp
    W[ndim] *= 1.0 + 0.3 * ramp
    q = o.prim_to_cons(W)
    Wr = o.cons_to_prim(q)
    dt = 0.3 * o.dt(q, 1.0)
    a = 0.25
    qa = o.stage(1, dt, q, q)
    dxs = w.dx[:ndim]
    cell_vol = float(np.prod(dxs))
    change = (qa - q).reshape(w.nvar, -1).sum(axis=1) * cell_vol
    Fhi = _euler_flux(o, Wr[:, :, :, -1:], 0).reshape(w.nvar, -1).sum(axis=1)
    Flo = _euler_flux(o, Wr[:, :, :, :1], 0).reshape(w.nvar, -1).sum(axis=1)
    face_area = cell_vol / dxs[0]
    expect = -a * dt * (Fhi - Flo) * face_area
    scale = np.abs(q).reshape(w.nvar, -1).max(axis=1) * cell_vol * q[0].size
    assert np.all(np.abs(change - expect) <= 1e-12 * scale), (change, expect)
    # the boundary fluxes stand well above the tolerance
    assert np.all(np.abs(expect[[0, 1, 1 + ndim]]) > 1e-8 * scale[[0, 1, 1 + ndim]])


def test_outflow_equals_domain_extended_by_edge_copies():
    """Both ghost layers of a zero-gradient side equal the edge cell: a
    domain extended by two real cells holding copies of the edge cells gives
    the same stage on the original cells.  App. D mode and CSF make the
    stage read the second ghost layer (D.1 central values, Delta^3 p, the
    sensor and the smoothing)."""
    w = wl.random_state(n=(14, 12), ncomp=3, iles=1, sigma=5.0, bc=[[O_, O_], [O_, O_], [P_, P_]])
    o = oracle.Oracle(w)
    q = o.prim_to_cons(w.primitives())
    qe = q
    we = w
    for d in range(2):
        ax = _axis(d)
        lo = np.repeat(np.take(qe, [0], axis=ax), 2, axis=ax)
        hi = np.repeat(np.take(qe, [qe.shape[ax] - 1], axis=ax), 2, axis=ax)
        qe = np.concatenate([lo, qe, hi], axis=ax)
        we = _resize(we, d, we.n[d] + 4, (O_, O_))
    oe = oracle.Oracle(we)
    dt = 0.3 * o.dt(q, 1.0)
    got = o.stage(1, dt, q, q)
    ext = oe.stage(1, dt, qe, qe)[:, :, 2:-2, 2:-2]
    assert _rel_max(got, ext) == 0.0, _rel_max(got, ext)
    sens = oe.sensor(qe)
    assert 0 < sens.sum() < sens.size    # both branches of the switch occur


def test_uniform_flow_through_outflow_stays_uniform():
    """A uniform state is a steady solution with zero-gradient boundaries."""
    w = wl.random_state(n=(16, 12), bc=[[O_, O_], [O_, O_], [P_, P_]])
    o = oracle.Oracle(w)
    W = np.zeros((w.nvar, 1, 12, 16))
    W[0], W[1], W[2], W[3], W[4] = 120.0, -35.0, 2e6, 320.0, 0.7
    q = o.prim_to_cons(W)
    q1, _ = o.step(q, 5, w.cfl)
    assert _rel_max(q1, q) <= 1e-13


def _inflow_case(ndim):
    if ndim == 2:
        n, bc = (10, 16), [[I_, O_], [P_, P_], [P_, P_]]
    else:
        n, bc = (6, 12, 12), [[I_, O_], [P_, P_], [P_, P_]]
    w = wl.random_state(n=n, ndim=ndim, bc=bc)
    hi = w.hi
    radius = 4.2 * w.dx[1]
    inflow = dict(yc=w.lo[1] + 0.5 * (hi[1] - w.lo[1]) + 0.3 * w.dx[1],
                  zc=w.lo[2] + 0.5 * (hi[2] - w.lo[2]), radius=radius, T=363.0, Y=[0.0],
                  u0=(300.0, 12.0, -7.0))
    return dataclasses.replace(w, inflow=inflow)


def _in_disc(w, j, k):
    f = w.inflow
    y = w.lo[1] + (j + 0.5) * w.dx[1] - f["yc"]
    z = (w.lo[2] + (k + 0.5) * w.dx[2] - f["zc"]) if w.ndim == 3 else 0.0
    return y * y + z * z <= f["radius"] ** 2


@pytest.mark.parametrize("ndim", [2, 3])
def test_inflow_disc_ghost_state(ndim):
    """Inflow disc on x-low: inside the disc (cell centres within the
    radius) the ghosts hold the Dirichlet u, T, Y with the edge cell's p
    (zero gradient); outside it the side is a slip wall.  With a uniform
    interior both ghost layers equal that state G, the boundary face's
    reconstructions return G and the interior state W (Sec. 3.3), and the
    first cell changes by -a dt (F_E(W) - F(G, W)) / dx with F the face flux
    of Eq. 3-1/3-2 (pinned elsewhere)."""
    w = _inflow_case(ndim)
    o = oracle.Oracle(w)
    nd = ndim
    Wc = np.array([20.0, 5.0, -3.0][:nd] + [2e6, 320.0, 0.9])
    W = np.broadcast_to(Wc[:, None, None, None], (w.nvar, w.n[2], w.n[1], w.n[0])).copy()
    q = o.prim_to_cons(W)
    Wr = o.cons_to_prim(q)[:, 0, 0, 0]
    dt = 0.3 * o.dt(q, 1.0)
    qa = o.stage(1, dt, q, q)
    FW = o.face_flux(0, [Wr] * 4)
    f = w.inflow
    n_in = 0
    for k in range(w.n[2]):
        for j in range(w.n[1]):
            if _in_disc(w, j, k):
                G = np.concatenate([np.array(f["u0"][:nd]), [Wr[nd], f["T"]], f["Y"][:w.ncomp - 1]])
                n_in += 1
            else:
                G = Wr.copy()
                G[0] = -G[0]
            Fin = o.face_flux(0, [G, G, Wr, Wr])
            expect = q[:, k, j, 0] - 0.25 * dt / w.dx[0] * (FW - Fin)
            got = qa[:, k, j, 0]
            assert np.all(np.abs(got - expect) <= 1e-13 * np.abs(q[:, 0, 0, 0]).max()), (j, k, got, expect)
            # away from x-low the uniform state stays as it is
            assert np.all(qa[:, k, j, 2:] == q[:, k, j, 2:])
    assert 0 < n_in < w.n[1] * w.n[2]


@pytest.mark.parametrize("kind", ["liquid_jet", "smooth_gas"])
def test_inflow_equals_domain_extended_by_ghost_states(kind):
    """Both ghost layers of the inflow side, on a non-uniform state: a
    domain extended by two real columns holding the Dirichlet state (inside
    the disc, with the first interior column's p) or the wall's mirror image
    (outside) gives the same first stage on the original cells, App. D and
    CSF included.  "smooth_gas" feeds gas matching the interior, so that the
    App. D switch takes the central branch (D.1, D.5, D.6) at the inflow
    face and the second ghost layer enters the face values."""
    w = _inflow_case(2)
    o0 = oracle.Oracle(w)
    W0 = o0.cons_to_prim(o0.prim_to_cons(w.primitives()))
    inflow = dict(w.inflow)
    if kind == "smooth_gas":
        inflow.update(T=float(W0[3, 0, :, 0].mean()), Y=[1.0],
                      u0=(float(W0[0, 0, :, 0].mean()), float(W0[1, 0, :, 0].mean()), 0.0))
    w = dataclasses.replace(w, inflow=inflow, scheme=dict(w.scheme, iles=1, sigma=5.0))
    o = oracle.Oracle(w)
    q = o.prim_to_cons(w.primitives())
    W = o.cons_to_prim(q)
    nd, f = 2, w.inflow
    ext = np.zeros((w.nvar, 1, w.n[1], 2))
    for j in range(w.n[1]):
        if _in_disc(w, j, 0):
            G = np.concatenate([np.array(f["u0"][:nd]), [W[nd, 0, j, 0], f["T"]], f["Y"][:w.ncomp - 1]])
            ext[:, 0, j, 0] = G
            ext[:, 0, j, 1] = G
        else:
            for m in range(2):      # ghost -1-m mirrors interior m
                g = W[:, 0, j, m].copy()
                g[0] = -g[0]
                ext[:, 0, j, 1 - m] = g
    we = _resize(w, 0, w.n[0] + 2, (O_, O_))
    oe = oracle.Oracle(we)
    qe = np.concatenate([oe.prim_to_cons(np.concatenate([ext, W], axis=3))[:, :, :, :2], q], axis=3)
    dt = 0.3 * o.dt(q, 1.0)
    got = o.stage(1, dt, q, q)
    ref = oe.stage(1, dt, qe, qe)[:, :, :, 2:]
    assert _rel_max(got, ref) <= 1e-11, _rel_max(got, ref)
    assert _rel_max(got, q) > 1e-6
    if kind == "smooth_gas":
        fl = oe.sensor(qe)[0]
        face = np.maximum(fl[:, 1], fl[:, 2])
        disc = np.array([_in_disc(w, j, 0) for j in range(w.n[1])])
        assert (face[disc] == 0).any()


@pytest.mark.parametrize("ndim", [2, 3])
def test_inflow_disc_per_cell_velocity(ndim):
    """The inflow disc with a velocity given per boundary cell (the jet's
    perturbed inflow): the ghost of boundary row (j, k) takes component a
    from in_u[a, k, j]; the first interior cell then changes by
    -a dt (F_E(W) - F(G, W)) / dx as for the uniform disc."""
    w = _inflow_case(ndim)
    nd = ndim
    rng = np.random.default_rng(60 + ndim)
    in_u = np.zeros((nd, w.n[2], w.n[1]))
    for a in range(nd):
        in_u[a] = (300.0 if a == 0 else 0.0) + rng.uniform(-20.0, 20.0, size=(w.n[2], w.n[1]))
    o = oracle.Oracle(w, inflow_u=in_u)
    Wc = np.array([20.0, 5.0, -3.0][:nd] + [2e6, 320.0, 0.9])
    W = np.broadcast_to(Wc[:, None, None, None], (w.nvar, w.n[2], w.n[1], w.n[0])).copy()
    q = o.prim_to_cons(W)
    Wr = o.cons_to_prim(q)[:, 0, 0, 0]
    dt = 0.3 * o.dt(q, 1.0)
    qa = o.stage(1, dt, q, q)
    FW = o.face_flux(0, [Wr] * 4)
    f = w.inflow
    n_in = 0
    for k in range(w.n[2]):
        for j in range(w.n[1]):
            if not _in_disc(w, j, k):
                continue
            n_in += 1
            G = np.concatenate([in_u[:, k, j], [Wr[nd], f["T"]], f["Y"][:w.ncomp - 1]])
            Fin = o.face_flux(0, [G, G, Wr, Wr])
            expect = q[:, k, j, 0] - 0.25 * dt / w.dx[0] * (FW - Fin)
            assert np.all(np.abs(qa[:, k, j, 0] - expect) <= 1e-13 * np.abs(q[:, 0, 0, 0]).max()), (j, k)
    assert n_in > 3


def test_inflow_disc_three_components():
    """The inflow disc with three components (the jet's N2, CH4 and liquid):
    inside the disc the ghosts take each tracked mass fraction of the
    inflow, in_Y[k] for component k."""
    w = wl.jet3d(n=(6, 12, 12), iles=0, sigma=0.0)
    w = dataclasses.replace(w, inflow=dict(w.inflow, Y=[0.2, 0.3], radius=4.2 * w.dx[1]))
    o = oracle.Oracle(w)
    nd = 3
    Wc = np.array([20.0, 5.0, -3.0, 6e6, 900.0, 0.7, 0.1])
    W = np.broadcast_to(Wc[:, None, None, None], (w.nvar, w.n[2], w.n[1], w.n[0])).copy()
    q = o.prim_to_cons(W)
    Wr = o.cons_to_prim(q)[:, 0, 0, 0]
    dt = 0.3 * o.dt(q, 1.0)
    qa = o.stage(1, dt, q, q)
    FW = o.face_flux(0, [Wr] * 4)
    f = w.inflow
    n_in = 0
    for k in range(w.n[2]):
        for j in range(w.n[1]):
            if not _in_disc(w, j, k):
                continue
            n_in += 1
            G = np.concatenate([np.array(f["u0"][:nd]), [Wr[nd], f["T"]], [0.2, 0.3]])
            Fin = o.face_flux(0, [G, G, Wr, Wr])
            expect = q[:, k, j, 0] - 0.25 * dt / w.dx[0] * (FW - Fin)
            assert np.all(np.abs(qa[:, k, j, 0] - expect) <= 1e-13 * np.abs(q[:, 0, 0, 0]).max()), (j, k)
    assert n_in > 3
