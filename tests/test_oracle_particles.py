"""Pins of the oracle's fluid-particle coupling (Sec. V A-C, E)."""
import math

import numpy as np

import oracle as O


def test_solid_marking_brute_force():
    """A node is inside particle p iff |x - x_p|^2 < R_p^2 (minimum image)."""
    nx, ny, nz = 20, 18, 16
    s = O.OracleSim(nx, ny, nz, wall_z0=1)
    xp, R = (18.3, 2.7, 7.1), 4.6  # straddles the periodic x and y boundaries
    s.add_particle(xp, R, kinematic=True)
    own = s.owner().reshape(nz, ny, nx)
    for z in range(nz):
        for y in range(ny):
            for x in range(nx):
                if z == 0:
                    assert own[z, y, x] == 1
                    continue
                d = [(x - xp[0] + nx / 2) % nx - nx / 2, (y - xp[1] + ny / 2) % ny - ny / 2, z - xp[2]]
                inside = d[0] ** 2 + d[1] ** 2 + d[2] ** 2 < R * R
                assert own[z, y, x] == (2 if inside else 0)


def test_sphere_in_fluid_at_rest_feels_no_force():
    n = 20
    s = O.OracleSim(n, n, n)
    s.init_fields(np.ones(n ** 3))
    s.add_particle((10.0, 10.0, 10.0), 5.0, kinematic=True)
    s.step(3)
    P = s.particles()[0]
    assert np.abs(P[0:6]).max() < 1e-13  # F_eta, T_eta: rounding of ~10^3 link terms
    assert np.abs(P[6:12]).max() == 0.0  # no interface: no capillary force


def test_momentum_exchange_balances_fluid_momentum():
    """Fixed sphere in a body-force driven flow: the fluid momentum changes per step
    by N_fluid g - F_eta exactly (momentum exchange = momentum the links remove)."""
    n, g = 18, 2e-5
    s = O.OracleSim(n, n, n, body_force_a=(g, 0.5 * g, 0.0), body_force_b=(g, 0.5 * g, 0.0), sigma=0.0)
    s.init_fields(np.ones(n ** 3))
    s.add_particle((8.3, 9.1, 8.6), 4.4, kinematic=True)
    nfluid = int((s.owner() == 0).sum())
    s.step(30)
    P0 = s.diag()[4:7]
    for _ in range(5):
        s.step(1)
        P1 = s.diag()[4:7]
        Feta = s.particles()[0][0:3]
        expect = nfluid * np.array([g, 0.5 * g, 0.0]) - Feta
        assert np.abs((P1 - P0) - expect).max() < 1e-12 * max(1.0, np.abs(Feta).max())
        assert np.abs(Feta).max() > 1e-4  # the flow does load the sphere
        P0 = P1


def test_moving_sphere_mass_bookkeeping():
    """Kinematic sphere crossing nodes: total mass changes by bounce-back source +
    refilled mass - covered mass, step by step (Sec. V A, V C)."""
    n = 20
    s = O.OracleSim(n, n, n, sigma=0.0)
    s.init_fields(np.ones(n ** 3))
    s.add_particle((6.2, 10.0, 10.0), 3.7, v=(0.21, 0.07, 0.0), kinematic=True)
    s.step(1)
    M0 = s.diag()[3]
    seen_refill = seen_cover = False
    for _ in range(25):
        s.step(1)
        d = s.diag()
        assert abs(d[3] - (M0 + d[0] + d[1] - d[2])) < 1e-12 * M0
        seen_refill |= d[1] > 0
        seen_cover |= d[2] > 0
        M0 = d[3]
    assert seen_refill and seen_cover


def test_capillary_symmetric_interface_zero_force():
    """Sphere centred on a flat interface, 90 deg: the force cancels by symmetry."""
    n = 33
    z = np.arange(n, dtype=float)
    phi = np.broadcast_to(np.tanh(0.5 * (z - 16.0))[:, None, None], (n, n, n)).reshape(-1)
    s = O.OracleSim(n, n, n, sigma=0.01)
    s.init_fields(phi)
    s.add_particle((16.0, 16.0, 16.0), 8.0, theta_deg=90.0, kinematic=True)
    s.eval_interface()
    F, T, used = s.capillary(0)
    assert used > 0
    scale = 0.01 * 8.0
    assert np.abs(F).max() < 1e-12 * scale
    assert np.abs(T).max() < 1e-12 * scale * 8.0


def test_capillary_matches_surface_integral():
    """Sec. V F: the Lagrangian-point sum approximates
    C sigma oint (1 - phi^2) [n_s - (n.n_s) n] dA over the sphere, evaluated here by
    brute-force quadrature of the analytic field of a spherical drop crossing the
    particle (wetting rotation disabled so the gradient is the plain stencil)."""
    n, a, Rd, Rp, sigma, C = 48, 0.5, 14.0, 10.0, 0.01, 1.0
    xd = np.array([n / 2, n / 2, n / 2 - 5.0])
    xp = np.array([n / 2, n / 2, n / 2 - 5.0 + Rd + 0.3 * Rp])
    z, y, x = np.meshgrid(*(np.arange(n),) * 3, indexing="ij")
    r = np.sqrt((x - xd[0]) ** 2 + (y - xd[1]) ** 2 + (z - xd[2]) ** 2)
    s = O.OracleSim(n, n, n, sigma=sigma, cap_norm=C, wet_phi_max=0.0)
    s.init_fields(np.tanh(a * (Rd - r)).reshape(-1))
    s.add_particle(xp, Rp, kinematic=True)
    s.eval_interface()
    F, T, _ = s.capillary(0)
    na = nv = 720
    al = (np.arange(na) + 0.5) * math.pi / na
    vp = np.arange(nv) * 2 * math.pi / nv
    A, V = np.meshgrid(al, vp, indexing="ij")
    ns = np.stack([np.sin(A) * np.cos(V), np.sin(A) * np.sin(V), np.cos(A)], -1)
    d = xp + Rp * ns - xd
    rr = np.linalg.norm(d, axis=-1)
    ph = np.tanh(a * (Rd - rr))
    nh = -d / rr[..., None]
    m = ns - (nh * ns).sum(-1)[..., None] * nh
    dA = Rp ** 2 * np.sin(A) * (math.pi / na) * (2 * math.pi / nv)
    Fb = ((C * sigma * (1 - ph ** 2) * dA)[..., None] * m).sum((0, 1))
    assert Fb[2] < 0  # the drop below pulls the particle down along the line of centres
    assert abs(F[2] / Fb[2] - 1) < 0.05
    assert np.abs(F[:2]).max() < 1e-12 and np.abs(T).max() < 1e-12


# ---------------------------------------------------------------------------
# Pins of the refill values, the momentum-exchange torque and the sphere branch
# of the wetting normal.  Each one recomputes the quantity from the paper's
# definition with this file's own lattice arithmetic (velocities and weights
# from |c|^2, pinned in test_oracle_lattice.py) and the oracle's state.
# ---------------------------------------------------------------------------
def _lat():
    c, w, _ = O.lattice()
    return c, w


def _feq(rho, u, c, w):
    """Second-order equilibrium of Sec. V C: w_i rho (1 + 3 c.u + 9/2 (c.u)^2 - 3/2 u^2)."""
    cu = c @ u
    return w * rho * (1.0 + 3.0 * cu + 4.5 * cu * cu - 1.5 * (u @ u))


def _nbr(n3, z, y, x, d):
    nx, ny, nz = n3
    return (((z + d[2]) % nz) * ny + (y + d[1]) % ny) * nx + (x + d[0]) % nx


def _refill_expected(s, own0, c, w, xp, vp, wp):
    """Sec. V C refill of every node that the particle uncovered in the last
    step: f^{a,b}_eq(rho_bar^{a,b}, u_p + w_p x (x - x_p)), rho_bar the mean
    density over the moving-direction neighbours that are fluid and were not
    fresh (two hops along the same directions if there is none, the ambient
    state (0, rho0) if there is still none; reading c16)."""
    n3 = (s.nx, s.ny, s.nz)
    own1 = s.owner()
    fa, fb = s.pops()
    fresh = (own0 >= 2) & (own1 == 0)
    out, branch = [], []
    for g in np.nonzero(fresh)[0]:
        z, y, x = g // (s.nx * s.ny), (g // s.nx) % s.ny, g % s.nx
        for hop in (1, 2):
            src = [q for q in (_nbr(n3, z, y, x, hop * c[i]) for i in range(1, 19)) if own1[q] == 0 and not fresh[q]]
            if src:
                break
        if src:
            ra = np.mean([fa[:, q].sum() for q in src])
            rb = np.mean([fb[:, q].sum() for q in src])
            branch.append(hop)
        else:
            ra, rb = 0.0, s.params.rho0
            branch.append(0)
        d = np.array([x, y, z], float) - xp
        d -= np.array(n3) * np.round(d / np.array(n3))
        u = vp + np.cross(wp, d)
        out.append((g, _feq(ra, u, c, w), _feq(rb, u, c, w)))
    return out, branch, fa, fb


def test_refill_values_from_the_neighbour_mean():
    """Sec. V C: a fast kinematic sphere over a fluid of random density and order
    parameter; every uncovered node holds f_eq of the mean over its fluid,
    non-fresh neighbours (N_f of them, not 18) at the rigid-body velocity of its
    own position, including nodes that need the two-hop fallback."""
    c, w = _lat()
    n = 22
    rng = np.random.default_rng(11)
    s = O.OracleSim(n, n, n, sigma=0.01)
    s.init_fields(rng.uniform(-0.9, 0.9, n ** 3), rng.uniform(0.9, 1.1, n ** 3))
    vp, wp = np.array([2.2, 0.4, 0.1]), np.array([0.01, -0.02, 0.015])
    s.add_particle((6.3, 11.2, 10.7), 4.3, v=vp, w=wp, kinematic=True)
    seen = set()
    checked = 0
    for _ in range(3):
        own0 = s.owner().copy()
        s.step(1)
        xp = s.particles()[0][18:21]
        exp, branch, fa, fb = _refill_expected(s, own0, c, w, xp, vp, wp)
        seen |= set(branch)
        for g, ea, eb in exp:
            # at |u| ~ 2 the polynomial's terms reach ~10 and cancel: 1e-13 absolute
            assert np.abs(fa[:, g] - ea).max() < 1e-13 and np.abs(fb[:, g] - eb).max() < 1e-13
            checked += 1
    assert checked > 100 and {1, 2} <= seen


def test_refill_ambient_without_fluid_neighbours():
    """Reading c16's last fallback: a sphere in a cavity that holds no fluid at
    all leaves behind nodes with no fluid within two hops; they take
    f_eq(0, u) for phase a and f_eq(rho0, u) for phase b."""
    c, w = _lat()
    n = 20
    xp0, R = np.array([9.4, 10.1, 9.8]), 4.2
    z, y, x = np.meshgrid(*(np.arange(n),) * 3, indexing="ij")
    inside = (x - xp0[0]) ** 2 + (y - xp0[1]) ** 2 + (z - xp0[2]) ** 2 < R * R
    s = O.OracleSim(n, n, n, sigma=0.0, rho0=1.3)
    s.set_static_solid(~inside)
    s.init_fields(np.ones(n ** 3))
    vp, wp = np.array([1.1, -0.3, 0.2]), np.array([0.0, 0.02, -0.01])
    s.add_particle(xp0, R, v=vp, w=wp, kinematic=True)
    own0 = s.owner().copy()
    s.step(1)
    exp, branch, fa, fb = _refill_expected(s, own0, c, w, s.particles()[0][18:21], vp, wp)
    assert len(exp) > 10 and set(branch) == {0}
    for g, ea, eb in exp:
        assert np.abs(fa[:, g]).max() == 0.0
        assert np.abs(fb[:, g] - eb).max() < 1e-15


def test_torque_balances_fluid_angular_momentum():
    """Sec. V B: a kinematically spinning sphere that straddles the periodic
    boundary, in fluid that starts at rest.  Per link the fluid gains
    (x - x_p) x c_i (f_in + f_out) and the particle receives
    (x_w - x_p) x [(c_out - u_w) f_out - (c_in - u_w) f_in], x_w the link
    midpoint; since c_i x c_i = 0 the two differ only by
    (x_w - x_p) x u_w (f_in - f_out), f_in - f_out = 6 w_i rho c_i.u_w.  So
    T_eta = -dL_fluid + sum_links (x_w - x_p) x u_w 6 w_i rho c_i.u_w, with the
    fluid's angular momentum L about x_p (minimum image) before and after the
    step.  The disturbance reaches no far periodic boundary within the steps
    checked, so L has no boundary flux."""
    c, w = _lat()
    n = 26
    s = O.OracleSim(n, n, n, sigma=0.0)
    s.init_fields(-np.ones(n ** 3))
    xp, R = np.array([1.3, 12.7, 11.9]), 4.6
    om = np.array([0.004, -0.007, 0.011])
    s.add_particle(xp, R, w=om, kinematic=True)
    z, y, x = np.meshgrid(*(np.arange(n),) * 3, indexing="ij")
    pos = np.stack([x.ravel(), y.ravel(), z.ravel()]).astype(float)

    def mi(d):
        return d - n * np.round(d / n)

    r = mi(pos - xp[:, None])

    def ang(own):
        fa, fb = s.pops()
        f = fa + fb
        m = own == 0
        return np.cross(r[:, m].T, (c.T @ f)[:, m].T).sum(0), f.sum(0)

    def link_term(own, rho, lever_at_node=False):
        C = np.zeros(3)
        for i in range(1, 19):
            src = ((((z - c[i, 2]) % n) * n + (y - c[i, 1]) % n) * n + (x - c[i, 0]) % n).ravel()
            idx = np.nonzero((own == 0) & (own[src] >= 2))[0]
            lev = mi(pos[:, idx] - 0.5 * c[i][:, None] - xp[:, None])
            uw = np.cross(om, lev.T).T
            d = 6.0 * w[i] * rho[idx] * (c[i] @ uw)
            C += (np.cross((r[:, idx] if lever_at_node else lev).T, uw.T) * d[:, None]).sum(0)
        return C

    s.step(1)
    for _ in range(4):
        own = s.owner()
        L0, rho = ang(own)
        C = link_term(own, rho)
        s.step(1)
        assert (s.owner() == own).all()
        L1, _ = ang(own)
        T = s.particles()[0][3:6]
        assert np.abs(T).max() > 1.0
        assert np.abs(T - (C - (L1 - L0))).max() < 1e-12 * np.abs(T).max()
        # the lever at the node instead of the link midpoint would miss by far more
        assert np.abs(link_term(own, rho, True) - C).max() > 1e-6


def test_sphere_wetting_normal_geometry():
    """Sec. V E with reading c11/c12 on spheres: two spheres of different contact
    angle across a flat diffuse interface, 0.7 lu apart.  At every fluid node
    next to a particle with |phi| < 0.99, -grad(phi) after the wetting step has
    the magnitude of the plain stencil gradient and the direction
    cos(theta_p) n_s + sin(theta_p) e, where n_s = (x - x_p)/|x - x_p| of the
    nearest sphere surface, theta_p that sphere's angle and e the unit part of
    n* = -g/|g| normal to n_s (the candidate on n*'s side).  Every other node
    keeps the plain gradient."""
    n = 36
    zc = np.arange(n, dtype=float)
    phi = np.broadcast_to(np.tanh(0.55 * (17.3 - zc))[:, None, None], (n, n, n)).reshape(-1)
    sph = [((11.4, 17.2, 18.1), 6.3, 40.0), ((24.3, 18.4, 16.9), 6.0, 125.0)]
    grads = []
    for wet in (0.99, 0.0):
        s = O.OracleSim(n, n, n, sigma=0.01, wet_phi_max=wet)
        s.init_fields(phi)
        for xp, R, th in sph:
            s.add_particle(xp, R, theta_deg=th, kinematic=True)
        ph, g = s.eval_interface()
        grads.append(g)
        own = s.owner()
    g1, g0 = grads
    c, _ = _lat()
    n3 = (n, n, n)
    rotated = nearest_used = 0
    for gi in np.nonzero(own == 0)[0]:
        z, y, x = gi // (n * n), (gi // n) % n, gi % n
        owners = {own[_nbr(n3, z, y, x, c[i])] for i in range(1, 19)} - {0}
        if not owners or abs(ph[gi]) >= 0.99:
            assert np.array_equal(g1[:, gi], g0[:, gi])
            continue
        dist = []
        for o in sorted(owners):
            xp, R, th = sph[o - 2]
            d = np.array([x, y, z], float) - np.array(xp)
            dist.append((np.linalg.norm(d) - R, o - 2, d / np.linalg.norm(d), math.radians(th)))
        _, p, ns, th = min(dist)
        nearest_used += len(owners) > 1
        gm = np.linalg.norm(g0[:, gi])
        nst = -g0[:, gi] / gm
        e = nst - (nst @ ns) * ns
        if np.linalg.norm(e) < 1e-3:
            continue
        e /= np.linalg.norm(e)
        expect = -gm * (math.cos(th) * ns + math.sin(th) * e)
        assert np.abs(g1[:, gi] - expect).max() < 1e-12 * max(gm, 1e-3)
        rotated += 1
    assert rotated > 100 and nearest_used > 0
