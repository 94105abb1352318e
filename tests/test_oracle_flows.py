"""Pins of the oracle's whole time step against closed-form flows.

 - without bodies the scheme is the textbook fractional step (Section 2):
   the no-slip shear wave and the x-y Taylor-Green vortex (free-slip walls)
   decay as their closed forms, at second order in the grid spacing;
 - the IB interpolation of Eq. new_IB is exact for fields linear along the
   wall normal: an immersed plane moving tangentially between two resting
   walls carries the exact piecewise-linear Couette profile;
 - an immersed plane splitting a channel driven by a uniform force recovers
   the two Poiseuille profiles at second order (Section 4.2's claim);
 - q makes the discrete divergence of the projected field equal q to
   machine precision and conserves mass (Eqs. mod_div, constraint_q);
 - Eq. new_IB reproduces affine fields exactly on the forcing nodes, and
   the no-slip error of Section 4.4 then vanishes.
"""
import numpy as np
import pytest

from oracle import oracle as orc
from oracle.oracle import OracleSim
from helpers import node_coords, sample, order
from paper_2606_09799_gb300 import inputs

PI = np.pi


def _plane(yw, lx, lz, vel=(0.0, 0.0, 0.0)):
    big = 0.25
    xyz = np.array([[-big * lx, yw, -big * lz], [(1 + big) * lx, yw, -big * lz],
                    [-big * lx, yw, (1 + big) * lz], [(1 + big) * lx, yw, (1 + big) * lz]])
    tri = np.array([[0, 1, 3], [0, 3, 2]], dtype=np.int32)
    return xyz, np.tile(np.asarray(vel, dtype=np.float64), (4, 1)), tri


@pytest.mark.parametrize("scheme", ["rk2", "ab"])
def test_shear_wave_decay_second_order(scheme):
    """u = sin(pi y) exp(-pi^2 t / Re), no-slip walls: advection vanishes,
    pressure stays zero."""
    re, T = 10.0, 0.05
    errs = []
    for ny in (16, 32):
        dt = 0.2 / ny
        nsteps = int(round(T / dt))
        sim = OracleSim(4, ny, 4, re=re, dt=dt, scheme=scheme)
        sim.u[...] = sample(sim.g, 0, lambda X, Y, Z: np.sin(PI * Y) + 0 * X)
        sim.step(nsteps)
        t = nsteps * dt
        ex = sample(sim.g, 0, lambda X, Y, Z: np.sin(PI * Y) * np.exp(-PI ** 2 * t / re) + 0 * X)
        errs.append(np.abs(sim.u - ex).max())
        assert np.abs(sim.v).max() < 1e-13 and np.abs(sim.w).max() < 1e-13
        assert np.abs(sim.p).max() < 1e-12
    assert order(*errs) > 1.8, errs


def test_taylor_green_free_slip_second_order():
    """u = sin(2 pi x) cos(pi y) F, v = -2 cos(2 pi x) sin(pi y) F,
    F = exp(-5 pi^2 t / Re), free-slip walls."""
    re, T = 20.0, 0.04
    errs, perr = [], []
    for n in (16, 32):
        dt = 0.16 / n
        nsteps = int(round(T / dt))
        sim = OracleSim(n, n, 2, lz=2.0 / n, re=re, dt=dt, ybc=1)
        g = sim.g
        sim.u[...] = sample(g, 0, lambda X, Y, Z: np.sin(2 * PI * X) * np.cos(PI * Y))
        sim.v[...] = sample(g, 1, lambda X, Y, Z: -2 * np.cos(2 * PI * X) * np.sin(PI * Y))
        sim.step(nsteps)
        t = nsteps * dt
        F = np.exp(-5 * PI ** 2 * t / re)
        eu = np.abs(sim.u - sample(g, 0, lambda X, Y, Z: np.sin(2 * PI * X) * np.cos(PI * Y) * F)).max()
        ev = np.abs(sim.v - sample(g, 1, lambda X, Y, Z: -2 * np.cos(2 * PI * X) * np.sin(PI * Y) * F)).max()
        errs.append(max(eu, ev))
        assert np.abs(sim.w).max() < 1e-13
        # pressure: p = (1/4)[cos(4 pi x) + 4 cos(2 pi y)] F^2 up to a constant (time-level
        # shifts make this first order in dt, so only its shape is checked loosely)
        pex = sample(g, 3, lambda X, Y, Z: 0.25 * (np.cos(4 * PI * X) + 4 * np.cos(2 * PI * Y)) * F ** 2)
        pex -= pex.mean()
        perr.append(np.abs(sim.p - sim.p.mean() - pex).max())
    assert order(*errs) > 1.8, errs
    assert perr[1] < 0.05 and perr[1] < perr[0], perr


def test_immersed_plane_couette_is_exact():
    """A plane at y_w moving at U_p in x between resting walls: the steady
    discrete solution is the exact piecewise-linear profile, because the
    linear reconstruction of Eq. new_IB and the second difference are exact
    for it."""
    yw, up, ny = 0.4137, 0.8, 16
    L = 4.0 / ny                                  # cubic cells, x and z invariant flow
    sim = OracleSim(4, ny, 4, lx=L, lz=L, re=1.0, dt=0.01)
    xyz, vel, tri = _plane(yw, L, L, (up, 0.0, 0.0))
    sim.set_surface(xyz, vel, tri)
    sim.step(300)
    Y = node_coords(sim.g, 0)[1]
    ex = np.where(Y < yw, up * Y / yw, up * (1 - Y) / (1 - yw))
    fluid = sim.owners[0] < 0
    err = np.abs(sim.u - ex)[fluid].max()
    assert err < 1e-10, err
    assert sim.last["slip"] < 1e-10


def _poiseuille(ny, use_q=True):
    yw, G, re = 0.4137, 1.0, 1.0
    L = 4.0 / ny
    sim = OracleSim(4, ny, 4, lx=L, lz=L, re=re, dt=0.01, use_q=use_q)
    xyz, vel, tri = _plane(yw, L, L)
    sim.set_surface(xyz, vel, tri)
    sim.set_body_force(G, 0.0, 0.0)
    sim.step(300)
    Y = np.broadcast_to(node_coords(sim.g, 0)[1], sim.u.shape)
    ex = np.where(Y < yw, 0.5 * G * re * Y * (yw - Y), 0.5 * G * re * (Y - yw) * (1 - Y))
    fluid = sim.owners[0] < 0
    up = fluid & (Y > yw)
    # Section 4.2: a 4th-order Chebyshev fit of the + side profile, extrapolated
    # to the immersed wall, measures the no-slip error there
    yy = np.broadcast_to(Y, sim.u.shape)[0, :, 0]
    sel = yy > yw
    coef = np.polynomial.chebyshev.chebfit(yy[sel], sim.u[0, sel, 0], 4)
    wall = abs(np.polynomial.chebyshev.chebval(yw, coef))
    return np.abs(sim.u - ex)[up].mean(), wall, sim


def test_immersed_plane_poiseuille_second_order():
    e = [_poiseuille(n) for n in (16, 32, 64)]
    l1 = [x[0] for x in e]
    wall = [x[1] for x in e]
    assert order(l1[0], l1[1]) > 1.7 and order(l1[1], l1[2]) > 1.7, l1
    assert order(wall[0], wall[1]) > 1.7 and order(wall[1], wall[2]) > 1.7, wall
    # steady parallel flow: q vanishes, the two elliptic equations coincide
    assert abs(e[-1][2].last["qF"]) < 1e-15


def test_projection_gives_div_equal_q_and_conserves_mass():
    wl = inputs.oscillating_sphere(n=32, steps=3, subdiv=2)
    sim = OracleSim(wl.nx, wl.ny, wl.nz, re=wl.re, dt=wl.dt)
    for s in range(wl.steps):
        xyz, vel = wl.surface(s)
        sim.set_surface(xyz, vel, wl.tri)
        sim.step()
        last = sim.last
        dV = sim.g.dx * sim.g.dy * sim.g.dz
        # Eq. constraint_q: sum_F q_F dV + sum_B q_B dV = 0
        assert abs(last["A"] + last["qF"] * last["VF"]) < 1e-14 * max(1.0, abs(last["A"]))
        assert sim.isb.sum() > 0
        d = orc.divergence(sim.g, sim.u, sim.v, sim.w)
        q = np.where(sim.isb == 1, last["div_hat"], last["qF"])
        assert np.abs(d - q).max() < 1e-11 / sim.g.dx
        assert abs((d * dV).sum()) < 1e-14


def test_without_q_divergence_is_zero():
    wl = inputs.oscillating_sphere(n=24, steps=2, subdiv=2)
    sim = OracleSim(wl.nx, wl.ny, wl.nz, re=wl.re, dt=wl.dt, use_q=False)
    for s in range(wl.steps):
        xyz, vel = wl.surface(s)
        sim.set_surface(xyz, vel, wl.tri)
        sim.step()
    d = orc.divergence(sim.g, sim.u, sim.v, sim.w)
    assert np.abs(d).max() < 1e-11 / sim.g.dx


def test_q_reduces_no_slip_error_on_moving_plate():
    """Section 4.4: with the modified elliptic equation the no-slip error on
    a moving zero-thickness plate is clearly smaller than with the standard
    one.  On this coarse 32^3 grid, once the impulsive-start transient has
    passed (steps 15-60), the mean error drops by well over 30% (the paper's
    developed flow on a finer grid shows about a factor 10)."""
    res = {}
    for use_q in (True, False):
        wl = inputs.heaving_plate(n=32, steps=60, nq=16)
        sim = OracleSim(wl.nx, wl.ny, wl.nz, re=wl.re, dt=4 * wl.dt, use_q=use_q)
        slips = []
        for s in range(wl.steps):
            xyz, vel = wl.surface_at(s * 4 * wl.dt)
            sim.set_surface(xyz, vel, wl.tri)
            sim.step()
            slips.append(sim.last["slip"])
        res[use_q] = np.mean(slips[15:])
    assert res[True] < 0.7 * res[False], res


def _affine(c):
    a = [0.3, -0.2, 0.5][c]
    B = np.array([[0.7, -1.1, 0.4], [0.2, 0.9, -0.6], [-0.5, 0.3, 1.2]])[c]
    return a, B


def test_forcing_exact_for_affine_fields():
    """Eq. new_IB with U = u(X) reproduces any affine field on the forcing
    nodes, on both sides of the surface; the no-slip error then vanishes."""
    g = orc.make_grid(24, 24, 24)
    xyz, tri = inputs.icosphere(3, 0.2, (0.49, 0.51, 0.5))
    diag = np.sqrt(g.dx ** 2 + g.dy ** 2 + g.dz ** 2)
    h = 2 * diag
    own, _ = orc.tag(g, xyz, tri)
    for c in range(3):
        a, B = _affine(c)
        fn = lambda X, Y, Z: a + B[0] * X + B[1] * Y + B[2] * Z
        f = sample(g, c, fn)
        vel = np.zeros_like(xyz)
        vel[:, c] = a + xyz @ B
        src = f.copy()
        dst = np.zeros_like(f)
        assert orc.force(g, c, src, dst, own[c], xyz, vel, tri, h) == 0
        m = own[c] >= 0
        np.testing.assert_allclose(dst[m], f[m], atol=1e-13)
        s, n = orc.ctypes.c_double(), orc.ctypes.c_long()
        orc.lib().orc_slip(orc.ctypes.byref(g), c, orc._p(f), orc._p(own[c]), orc._p(xyz), orc._p(vel),
                           orc._p(tri), h, orc.ctypes.byref(s), orc.ctypes.byref(n))
        assert n.value == m.sum() and s.value / n.value < 1e-13


@pytest.mark.parametrize("scheme", ["ab", "rk2"])
def test_gradient_mode_closed_form_pressure(scheme):
    """Closed form of one step from u^0 = eps G psi (psi a discrete Laplacian
    eigenvector, lambda = lx + ly + lz; free-slip walls keep every component of
    G psi an eigenvector of each 1-D operator).  Per sub-stage with p^s = P psi:
    R = dt[-alpha G p^s + alpha/Re L u^s] is a gradient, the approximate
    factorisation divides it by F = prod_d (1 + beta l_d), the projection
    removes it entirely (u^{s+1} = 0), and Eq. update_pressure gives
    p^{s+1} = p^s + phi (1 + beta lambda)."""
    g = orc.make_grid(8, 6, 4, 1.0, 1.0, 0.5, ybc=1)
    m, l, n = 1, 2, 1
    Z, Y, X = node_coords(g, 3)
    psi = np.ascontiguousarray(np.broadcast_to(
        np.cos(2 * PI * m * X / g.lx) * np.cos(PI * l * Y / g.ly) * np.cos(2 * PI * n * Z / g.lz),
        (g.nz, g.ny, g.nx)))
    lx = (2 - 2 * np.cos(2 * PI * m / g.nx)) / g.dx ** 2
    ly = (2 - 2 * np.cos(PI * l / g.ny)) / g.dy ** 2
    lz = (2 - 2 * np.cos(2 * PI * n / g.nz)) / g.dz ** 2
    lam = lx + ly + lz
    eps, re, dt = 1e-9, 3.0, 0.02
    sim = OracleSim(g.nx, g.ny, g.nz, g.lx, g.ly, g.lz, re=re, dt=dt, scheme=scheme, ybc=1)
    gu = (psi - np.roll(psi, 1, axis=2)) / g.dx
    gw = (psi - np.roll(psi, 1, axis=0)) / g.dz
    gv = np.zeros(orc.field_shape(g, 1))
    gv[:, 1:g.ny, :] = (psi[:, 1:, :] - psi[:, :-1, :]) / g.dy
    sim.u[...], sim.v[...], sim.w[...] = eps * gu, eps * gv, eps * gw
    sim.step(1)
    U, P = eps, 0.0          # u^s = U G psi, p^s = P psi
    for (gam, rho, alp) in orc.SCHEMES[scheme]:
        beta = alp * dt / (2 * re)
        F = (1 + beta * lx) * (1 + beta * ly) * (1 + beta * lz)
        # uhat = U G psi + (dt/F)(-alp P - alp/Re lam U) G psi = C G psi
        C = U + dt / F * (-alp * P - alp / re * lam * U)
        phi = C / (alp * dt)                 # L_c phi = D uhat / (alp dt) = -lam C psi / (alp dt)
        P = P + phi * (1 + beta * lam)
        U = 0.0
    scale = eps / dt
    assert np.abs(sim.u).max() < 1e-6 * eps * np.abs(gu).max()
    np.testing.assert_allclose(sim.p, P * psi, atol=1e-6 * scale)


def _energy_case(seed=3, n=12):
    """A small grid with a body (boundary cells) and random fields."""
    rng = np.random.default_rng(seed)
    g = orc.make_grid(n, n, n)
    xyz, tri = inputs.icosphere(2, 0.3, (0.5, 0.5, 0.5))
    own, _ = orc.tag(g, xyz, tri)
    isb = orc.boundary_cells(g, own)
    u, v, w, p = inputs.random_fields(n, n, n, seed)
    div = orc.divergence(g, u, v, w)
    return g, isb, u, v, w, p, div


def test_energy_q_satisfies_mass_and_energy_constraints():
    """App. B: the shape makes sum_F q dV + sum_B Du dV = 0 (mass) and
    sum_F (p - e) q dV + sum_B (p - e) Du dV = 0 (inviscid kinetic energy);
    e is |u|^2/2 with the velocity averaged to the cell centre (computed here
    independently of the oracle)."""
    g, isb, u, v, w, p, div = _energy_case()
    assert isb.sum() > 10
    q, coef = orc.q_energy(g, div, isb, p, u, v, w)
    dV = g.dx * g.dy * g.dz
    uc = 0.5 * (u + np.roll(u, -1, axis=2))
    vc = 0.5 * (v[:, :-1, :] + v[:, 1:, :])
    wc = 0.5 * (w + np.roll(w, -1, axis=0))
    pe = p - 0.5 * (uc ** 2 + vc ** 2 + wc ** 2)
    F, Bm = isb == 0, isb == 1
    np.testing.assert_array_equal(q[Bm], div[Bm])
    A = (div[Bm] * dV).sum()
    B = (pe[Bm] * div[Bm] * dV).sum()
    mass = (q[F] * dV).sum() + A
    energy = (pe[F] * q[F] * dV).sum() + B
    scale = np.abs(div).max() * dV * F.sum() * (1 + np.abs(pe).max())
    assert abs(mass) < 1e-13 * scale and abs(energy) < 1e-13 * scale
    assert abs(coef[1]) > 0          # the energy part is active


def test_energy_q_is_the_minimum_norm_field_of_the_two_constraints():
    """The Lagrangian of App. B: among all q on C_F meeting both constraints,
    the shape has the least sum q^2 dV -- the least-norm solution of the 2 x
    |C_F| linear system, computed here by numpy's least squares."""
    g, isb, u, v, w, p, div = _energy_case(seed=5)
    q, coef = orc.q_energy(g, div, isb, p, u, v, w)
    dV = g.dx * g.dy * g.dz
    uc = 0.5 * (u + np.roll(u, -1, axis=2))
    vc = 0.5 * (v[:, :-1, :] + v[:, 1:, :])
    wc = 0.5 * (w + np.roll(w, -1, axis=0))
    pe = p - 0.5 * (uc ** 2 + vc ** 2 + wc ** 2)
    F, Bm = isb == 0, isb == 1
    M = np.stack([np.full(F.sum(), dV), pe[F] * dV])
    rhs = -np.array([(div[Bm] * dV).sum(), (pe[Bm] * div[Bm] * dV).sum()])
    ref, *_ = np.linalg.lstsq(M, rhs, rcond=None)
    assert np.abs(q[F] - ref).max() < 1e-10 * np.abs(ref).max()


def test_energy_q_reduces_to_uniform_when_p_minus_e_is_uniform():
    g, isb, u, v, w, p, div = _energy_case(seed=7)
    z = [np.zeros_like(a) for a in (u, v, w)]
    q, coef = orc.q_energy(g, div, isb, np.full_like(p, 0.3), *z)
    _, qF, A, VF = orc.rhs_poisson(g, div, isb, 1, 1.0)
    assert coef[1] == 0.0
    np.testing.assert_allclose(q[isb == 0], qF, rtol=1e-15)


def test_energy_q_flow_projection_is_exact():
    """With the energy shape the projected field satisfies D u = q^k cell by
    cell to machine precision (Eq. mod_div with the App. B shape), and the
    total mass flux vanishes."""
    wl = inputs.oscillating_sphere(n=24, steps=3, subdiv=2)
    sim = OracleSim(wl.nx, wl.ny, wl.nz, re=wl.re, dt=wl.dt, use_q=2)
    for s in range(wl.steps):
        xyz, vel = wl.surface(s)
        sim.set_surface(xyz, vel, wl.tri)
        sim.step()
        d = orc.divergence(sim.g, sim.u, sim.v, sim.w)
        assert np.abs(d - sim.last["q_field"]).max() < 1e-11 / sim.g.dx
        assert abs((d * sim.g.dx * sim.g.dy * sim.g.dz).sum()) < 1e-14
        assert abs(sim.last["q_coef"][1]) > 0
