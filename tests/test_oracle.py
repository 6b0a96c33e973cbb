"""Pins of the FP64 oracle against what the paper and the mathematics fix.

Nothing here compares the oracle with itself: every check is a closed form,
an exact invariant, a special case with a textbook solution, a value the paper
prints (tests/golden/paper_constants.json), or an independently written
push-form update (brute force on tiny grids).  A dropped term, a wrong sign or
index, or a transposed operand anywhere in the oracle fails at least one test:

- lattice table / weights ........ isotropy moments to 4th order, paper weights
- equilibrium (Eq. (2)) .......... its 0th, 1st and 2nd moments in closed form
- bounce-back (Sec. 2.1) ......... Couette profile (sign and factor of the wall term),
                                   mass conservation, push-vs-pull brute force
- collision (Eq. (1), TRT) ....... shear-wave viscosity nu = (tau - 1/2)/3,
                                   Poiseuille exactness at Lambda = 3/16,
                                   TRT == BGK when Lambda = (tau - 1/2)^2
- forcing ........................ momentum grows by exactly F per cell and step,
                                   Poiseuille steady and start-up profiles
- pressure boundary .............. push-vs-pull, rest and uniform-flow fixed points,
                                   inlet/outlet channel (flux, profile, gradient)
- curved walls ................... off-grid Poiseuille at second order, q = 1/2 is
                                   half-way bounce-back, push-vs-pull brute force
- residuals ...................... closed values; uniform forced flow from rest
                                   (u_n = (n - 1/2) F exactly, so r = 1/(n - 1/2)
                                   and the stopping step in closed form); the
                                   period-2 mode cancels over an even interval
"""
import json
import os

import numpy as np
import pytest

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "paper_constants.json")


# ----------------------------------------------------------------- lattice
def test_lattice_matches_paper_weights_and_is_isotropic(orc):
    e, w, opp = orc.lattice()
    gold = json.load(open(GOLDEN))["d3q19_weights"]
    assert len(w) == gold["q"] == 19
    n2 = (e * e).sum(1)
    # 19 distinct velocities: the rest vector, 6 axis, 12 face diagonals
    assert len({tuple(v) for v in e}) == 19
    assert sorted(n2.tolist()) == [0] + [1] * 6 + [2] * 12
    frac = {0: gold["rest"], 1: gold["axis"], 2: gold["diagonal"]}
    for i in range(19):
        num, den = frac[int(n2[i])]
        assert w[i] == num / den
        assert (e[opp[i]] == -e[i]).all()
        assert opp[opp[i]] == i
    # lattice tensors: sum w = 1, sum w e = 0, sum w e e = 1/3 I,
    # sum w e_a e_b e_c = 0, sum w e_a e_b e_c e_d = (dd + dd + dd)/9
    d = np.eye(3)
    assert abs(w.sum() - 1) < 1e-15
    assert np.abs(w @ e).max() < 1e-15
    assert np.abs(np.einsum("i,ia,ib->ab", w, e, e) - d / 3).max() < 1e-15
    assert np.abs(np.einsum("i,ia,ib,ic->abc", w, e, e, e)).max() < 1e-15
    t4 = np.einsum("i,ia,ib,ic,id->abcd", w, e, e, e, e)
    iso = (np.einsum("ab,cd->abcd", d, d) + np.einsum("ac,bd->abcd", d, d)
           + np.einsum("ad,bc->abcd", d, d)) / 9
    assert np.abs(t4 - iso).max() < 1e-15
    # the direction numbering is the one documented in include/lbm.h
    assert e[1].tolist() == [1, 0, 0] and e[2].tolist() == [-1, 0, 0]
    assert e[7].tolist() == [1, 1, 0] and e[18].tolist() == [0, -1, 1]


def test_equilibrium_moments_closed_form(orc):
    """Eq. (2), shifted: sum feq = drho, sum e feq = rho0 u,
    sum e_a e_b feq = drho/3 d_ab + rho0 u_a u_b (incompressible model)."""
    gold = json.load(open(GOLDEN))["equilibrium_factors"]
    assert (gold["linear"], gold["quadratic"], gold["usq"]) == (3.0, 4.5, 1.5)
    e, w, _ = orc.lattice()
    rng = np.random.default_rng(7)
    for _ in range(20):
        drho = rng.uniform(-0.05, 0.05)
        u = rng.uniform(-0.1, 0.1, 3)
        rho0 = rng.uniform(0.5, 2.0)
        feq = orc.equilibrium(drho, u, rho0)
        assert abs(feq.sum() - drho) < 1e-15
        assert np.abs(e.T @ feq - rho0 * u).max() < 1e-15
        pi = np.einsum("i,ia,ib->ab", feq, e, e)
        assert np.abs(pi - (drho / 3 * np.eye(3) + rho0 * np.outer(u, u))).max() < 1e-15
        # against the unshifted form of Eq. (2) written out directly
        rho = rho0 + drho
        eu = e @ u
        full = w * (rho + rho0 * (3 * eu + 4.5 * eu**2 - 1.5 * u @ u))
        assert np.abs(full - w * rho0 - feq).max() < 1e-15
    assert np.all(orc.equilibrium(0.0, np.zeros(3), 1.0) == 0.0)


def test_collision_conserves_mass_and_adds_force(orc):
    """Collision keeps sum f and moves sum e f from rho0 u - F/2 to rho0 u + F/2."""
    rng = np.random.default_rng(3)
    e, _, _ = orc.lattice()
    for coll in (orc.BGK, orc.TRT):
        F = rng.uniform(-1e-3, 1e-3, 3)
        p = orc.Problem(dims=(1, 1, 1), tau=0.77, collision=coll, force=tuple(F))
        f = rng.uniform(-0.01, 0.01, 19)
        out, u = orc.collide(p, f)
        assert abs(out.sum() - f.sum()) < 1e-16
        assert np.abs(e.T @ f + F / 2 - u).max() < 1e-16
        assert np.abs(e.T @ out - (e.T @ f + F)).max() < 1e-16


def test_trt_reduces_to_bgk(orc):
    rng = np.random.default_rng(11)
    tau = 0.73
    f = rng.uniform(-0.02, 0.02, 19)
    kw = dict(dims=(1, 1, 1), tau=tau, force=(1e-4, -2e-4, 3e-4))
    a, _ = orc.collide(orc.Problem(collision=orc.BGK, **kw), f)
    b, _ = orc.collide(orc.Problem(collision=orc.TRT, magic=(tau - 0.5) ** 2, **kw), f)
    assert np.abs(a - b).max() < 1e-16
    c, _ = orc.collide(orc.Problem(collision=orc.TRT, magic=3 / 16, **kw), f)
    assert np.abs(a - c).max() > 1e-6  # Lambda matters when it differs


# ----------------------------------------------------------- fixed points
def _random_flags(rng, dims, frac=0.2, moving=True):
    nx, ny, nz = dims
    fl = (rng.random((nz, ny, nx)) < frac).astype(np.uint8)
    if moving:
        fl[(fl == 1) & (rng.random(fl.shape) < 0.3)] = 2
    return fl


def test_rest_state_is_bitwise_fixed_point(orc):
    rng = np.random.default_rng(1)
    dims = (7, 6, 5)
    p = orc.Problem(dims=dims, tau=0.6, flags=_random_flags(rng, dims, moving=False),
                    periodic=(1, 0, 0), collision=orc.TRT)
    f = orc.run(p, orc.zeros(p), 50)
    assert np.all(f == 0.0)


@pytest.mark.parametrize("coll", [0, 1])
def test_uniform_equilibrium_is_fixed_point(orc, coll):
    dims = (5, 4, 6)
    p = orc.Problem(dims=dims, tau=0.9, periodic=(1, 1, 1), collision=coll)
    u = np.array([0.02, -0.01, 0.03])
    rho = np.full(dims[::-1], 1.01)
    uu = np.broadcast_to(u[:, None, None, None], (3,) + dims[::-1])
    f0 = orc.init_equilibrium(p, rho, uu)
    f = orc.run(p, f0, 20)
    assert np.abs(f - f0).max() < 1e-15


# -------------------------------------------------------------- invariants
@pytest.mark.parametrize("coll", [0, 1])
def test_mass_conserved_in_closed_box_with_obstacles(orc, coll):
    rng = np.random.default_rng(5 + coll)
    dims = (8, 7, 6)
    p = orc.Problem(dims=dims, tau=0.7, flags=_random_flags(rng, dims, 0.15, moving=False),
                    collision=coll)
    f = rng.uniform(-1e-2, 1e-2, (19,) + dims[::-1]) * (p.flags == 0)
    m0, _ = orc.invariants(p, f)
    f = orc.run(p, f, 200)
    m1, _ = orc.invariants(p, f)
    assert abs(m1 - m0) / m0 < 1e-13


@pytest.mark.parametrize("coll", [0, 1])
def test_momentum_grows_by_force_each_step(orc, coll):
    rng = np.random.default_rng(9)
    dims = (6, 5, 4)
    F = np.array([2e-5, -1e-5, 3e-5])
    p = orc.Problem(dims=dims, tau=0.85, periodic=(1, 1, 1), collision=coll, force=tuple(F))
    f = rng.uniform(-1e-2, 1e-2, (19,) + dims[::-1])
    N = np.prod(dims)
    m_prev, j_prev = orc.invariants(p, f)
    for _ in range(10):
        f = orc.step(p, f)
        m, j = orc.invariants(p, f)
        assert abs(m - m_prev) < 1e-14 * m
        assert np.abs(j - j_prev - N * F).max() < 1e-13  # vs |N F| ~ 1e-3
        m_prev, j_prev = m, j


# ----------------------------------------------------- analytic profiles
@pytest.mark.parametrize("coll,tau", [(0, 0.8), (1, 0.65), (0, 1.5)])
def test_couette_profile_is_exact(orc, coll, tau):
    """Half-way walls at y=-1/2 (rest) and y=H-1/2 (moving with u_w along x):
    u_x(y) = u_w (y + 1/2)/H, exact for half-way bounce-back.  Pins the sign
    and the factor 6 w_i rho0 of the moving-wall term."""
    H, uw = 8, 0.01
    p = orc.Problem(dims=(2, H, 3), tau=tau, periodic=(1, 0, 1), collision=coll,
                    face_bc=(1, 1, 1, 2, 1, 1), wall_u=(uw, 0, 0))
    f = orc.run(p, orc.zeros(p), 8000)
    rho, u = orc.macroscopic(p, f)
    y = np.arange(H) + 0.5
    assert np.abs(u[0] - (uw * y / H)[None, :, None]).max() < 1e-14
    assert np.abs(u[1:]).max() < 1e-15
    assert np.abs(rho - 1).max() < 1e-13


def _poiseuille(F, nu, H):
    y = np.arange(H) + 0.5
    return F / (2 * nu) * y * (H - y)


def test_poiseuille_steady_trt_exact(orc):
    """TRT with Lambda = 3/16: half-way bounce-back reproduces the parabola
    u(y) = F/(2 nu) y (H - y) to roundoff, walls at y = -1/2 and H - 1/2."""
    H, F, tau = 16, 1e-5, 0.8
    p = orc.Problem(dims=(2, H, 2), tau=tau, periodic=(1, 0, 1), collision=orc.TRT,
                    magic=3 / 16, force=(F, 0, 0))
    f = orc.run(p, orc.zeros(p), 12000)
    _, u = orc.macroscopic(p, f)
    ua = _poiseuille(F, (tau - 0.5) / 3, H)
    assert np.abs(u[0, 0, :, 0] - ua).max() / ua.max() < 1e-12


def test_poiseuille_steady_bgk(orc):
    """BGK: exact at tau = 1/2 + sqrt(3)/4 (where (tau-1/2)^2 = 3/16); at other
    tau the profile carries a tau-dependent slip of a few 1e-3 relative."""
    H, F = 16, 1e-5
    tau = 0.5 + np.sqrt(3) / 4
    p = orc.Problem(dims=(2, H, 2), tau=tau, periodic=(1, 0, 1), force=(F, 0, 0))
    _, u = orc.macroscopic(p, orc.run(p, orc.zeros(p), 12000))
    ua = _poiseuille(F, (tau - 0.5) / 3, H)
    assert np.abs(u[0, 0, :, 0] - ua).max() / ua.max() < 1e-12
    p = orc.Problem(dims=(2, H, 2), tau=0.8, periodic=(1, 0, 1), force=(F, 0, 0))
    _, u = orc.macroscopic(p, orc.run(p, orc.zeros(p), 12000))
    err = np.abs(u[0, 0, :, 0] - _poiseuille(F, 0.1, H)).max() / _poiseuille(F, 0.1, H).max()
    assert 1e-4 < err < 1e-2


def test_poiseuille_startup_series(orc):
    """Start-up from rest: u(y,t) = F/(2nu) y(H-y)
    - sum_{n odd} 4 F H^2/(nu pi^3 n^3) sin(n pi y/H) exp(-nu n^2 pi^2 t/H^2)."""
    H, F, tau = 32, 1e-6, 0.8
    nu = (tau - 0.5) / 3
    p = orc.Problem(dims=(1, H, 1), tau=tau, periodic=(1, 0, 1), collision=orc.TRT,
                    force=(F, 0, 0))
    y = np.arange(H) + 0.5
    for t in (200, 1000):
        _, u = orc.macroscopic(p, orc.run(p, orc.zeros(p), t))
        ua = _poiseuille(F, nu, H)
        for n in range(1, 600, 2):
            ua = ua - 4 * F * H * H / (nu * np.pi**3 * n**3) * np.sin(n * np.pi * y / H) \
                * np.exp(-nu * n * n * np.pi**2 * t / H**2)
        assert np.abs(u[0, 0, :, 0] - ua).max() < 0.01 * ua.max()


@pytest.mark.parametrize("coll,tau", [(0, 0.8), (1, 0.6), (0, 1.2)])
def test_shear_wave_decays_at_lattice_viscosity(orc, coll, tau):
    """u_x = A sin(k y) in a periodic box decays as exp(-nu k^2 t) with
    nu = (tau - 1/2) c_s^2, c_s^2 = 1/3 (Sec. 2.1)."""
    L, A = 32, 1e-3
    p = orc.Problem(dims=(2, L, 2), tau=tau, periodic=(1, 1, 1), collision=coll)
    y = np.arange(L) + 0.5
    u0 = np.zeros((3, 2, L, 2))
    u0[0] = (A * np.sin(2 * np.pi * y / L))[None, :, None]
    f = orc.init_equilibrium(p, np.ones((2, L, 2)), u0)
    amp = []
    for t in (100, 600):
        _, u = orc.macroscopic(p, orc.run(p, f, t))
        amp.append((u[0, 0, :, 0] * np.sin(2 * np.pi * y / L)).sum() * 2 / L)
    k = 2 * np.pi / L
    nu = np.log(amp[0] / amp[1]) / (k * k * 500)
    assert abs(nu / ((tau - 0.5) / 3) - 1) < 0.01


# ------------------------------------------------------------ brute force
@pytest.mark.parametrize("seed", range(12))
def test_pull_step_matches_independent_push_step(orc, seed):
    """Random PDFs, random obstacles (resting and moving), random periodicity
    and wall kinds on 3^3..5^3 grids: the shifted pull step equals the
    unshifted push-and-reflect step written separately."""
    rng = np.random.default_rng(100 + seed)
    dims = tuple(int(v) for v in rng.integers(3, 6, 3))
    p = orc.Problem(dims=dims, tau=float(rng.uniform(0.55, 1.5)),
                    flags=_random_flags(rng, dims, 0.2),
                    periodic=tuple(int(v) for v in rng.integers(0, 2, 3)),
                    face_bc=tuple(int(v) for v in rng.integers(1, 3, 6)),
                    collision=int(seed % 2), magic=float(rng.uniform(0.05, 0.3)),
                    force=tuple(rng.uniform(-1e-3, 1e-3, 3)),
                    wall_u=tuple(rng.uniform(-0.05, 0.05, 3)))
    f = rng.uniform(-1e-2, 1e-2, (19,) + dims[::-1]) * (p.flags == 0)
    for _ in range(3):
        a = orc.step(p, f)
        b = orc.push_step(p, f)
        assert np.isfinite(b).all()
        assert np.abs(a - b).max() < 1e-14
        f = a


@pytest.mark.parametrize("seed", range(8))
def test_pull_step_matches_push_step_with_pressure_boundaries(orc, seed):
    """The same brute force with pressure cells and faces (anti-bounce-back,
    random rho_b): the pull rule in shifted variables equals the push rule
    2 w [rho_b + rho0 (4.5 (e.u)^2 - 1.5 u^2)] - f* written separately in
    unshifted ones."""
    rng = np.random.default_rng(300 + seed)
    dims = tuple(int(v) for v in rng.integers(3, 6, 3))
    fl = _random_flags(rng, dims, 0.25)
    fl[(fl != 0) & (rng.random(fl.shape) < 0.4)] = orc.PRESSURE
    p = orc.Problem(dims=dims, tau=float(rng.uniform(0.55, 1.5)), flags=fl,
                    periodic=tuple(int(v) for v in rng.integers(0, 2, 3)),
                    face_bc=tuple(int(v) for v in rng.integers(1, 4, 6)),
                    collision=int(seed % 2), magic=float(rng.uniform(0.05, 0.3)),
                    force=tuple(rng.uniform(-1e-3, 1e-3, 3)),
                    wall_u=tuple(rng.uniform(-0.05, 0.05, 3)), rho_b=float(rng.uniform(0.99, 1.01)))
    assert (p.flags == orc.PRESSURE).any()
    f = rng.uniform(-1e-2, 1e-2, (19,) + dims[::-1]) * (p.flags == 0)
    for _ in range(3):
        a = orc.step(p, f)
        b = orc.push_step(p, f)
        assert np.isfinite(b).all()
        assert np.abs(a - b).max() < 1e-14
        f = a


def test_velocity_inlet_pressure_outlet_channel(orc):
    """A velocity inlet (a moving-wall face at -x, Ladd bounce-back) and a
    pressure outlet (anti-bounce-back at +x, rho_b = rho0) on a channel with
    walls at -y/+y: the steady state carries the same mass flux through every
    cross-section, develops the Poiseuille profile 6 U_mean y (H - y) / H^2 and
    the density gradient -36 nu rho0 U_mean / H^2 (dp/dx = -12 mu U_mean / H^2,
    p = rho / 3), and the density next to the outlet is rho_b up to half a
    cell of that gradient."""
    orc.set_threads(os.cpu_count() or 1)
    nx, H, U, tau = 48, 12, 0.01, 0.8
    nu = (tau - 0.5) / 3
    p = orc.Problem(dims=(nx, H, 1), tau=tau, periodic=(0, 0, 1),
                    face_bc=(orc.MOVING, orc.PRESSURE, 1, 1, 1, 1), wall_u=(U, 0, 0), rho_b=1.0)
    f = orc.zeros(p)
    prev = None
    for _ in range(60):
        f = orc.run(p, f, 500)
        rho, u = orc.macroscopic(p, f)
        if prev is not None and np.abs(u - prev).max() < 1e-12:
            break
        prev = u
    orc.set_threads(1)
    flux = u[0].sum(axis=(0, 1))  # per x, summed over y and z
    assert np.abs(flux / flux.mean() - 1).max() < 1e-9
    U_mean = flux.mean() / H
    y = np.arange(H) + 0.5
    prof = u[0, 0, :, nx // 2]
    assert np.abs(prof - 6 * U_mean * y * (H - y) / H**2).max() < 1e-2 * prof.max()
    grad = np.gradient(rho[0, H // 2, :])[nx // 3: 2 * nx // 3].mean()
    want = -36 * nu * U_mean / H**2
    assert abs(grad / want - 1) < 2e-2
    # what remains is the non-equilibrium part the rule does not model (the
    # shear next to the outlet): 2.3 (1.5 U_mean)^2 here, 5.3 without the
    # velocity correction
    assert abs(rho[0, H // 2, -1] - (1.0 - 0.5 * grad)) < 3.0 * (1.5 * U_mean) ** 2


def test_pressure_boundary_passes_uniform_flow_exactly(orc):
    """A uniform equilibrium flow at density rho_b through pressure faces and
    past pressure cells is a fixed point to roundoff: the returning
    population -f*_i + 2 f_eq,sym_i equals f_eq,ibar exactly when the
    boundary velocity is the flow's.  A dropped or mis-signed velocity
    correction, a wrong 4.5 or 1.5, or a boundary velocity other than the
    cell's own drives the state away (by 2e-3 without the correction)."""
    rng = np.random.default_rng(9)
    dims = (7, 6, 5)
    fl = np.zeros(dims[::-1], np.uint8)
    fl[(rng.random(fl.shape) < 0.1)] = orc.PRESSURE
    rho_b, u = 1.003, np.array([0.03, -0.02, 0.01])
    e, w, _ = orc.lattice()
    for coll in (orc.BGK, orc.TRT):
        p = orc.Problem(dims=dims, tau=0.7, flags=fl, periodic=(0, 1, 1), face_bc=(3, 3, 1, 1, 1, 1),
                        collision=coll, rho_b=rho_b)
        eu = e @ u
        feq = w * ((rho_b - 1.0) + 3 * eu + 4.5 * eu**2 - 1.5 * u @ u)
        f = feq[:, None, None, None] * (fl == 0)
        g = orc.run(p, f.copy(), 30)
        assert np.abs(g - f).max() < 1e-16


def test_pressure_boundary_rest_state_is_a_fixed_point(orc):
    """At rest every term of the anti-bounce-back rule is exact: the state
    f~ = w drho_b (uniform density rho_b, u = 0) stays put to roundoff with
    pressure faces and pressure cells, which fixes the rule's sign and its
    factor 2 (any other would drive the density away from rho_b)."""
    rng = np.random.default_rng(8)
    dims = (9, 7, 5)
    fl = np.zeros(dims[::-1], np.uint8)
    fl[(rng.random(fl.shape) < 0.1)] = orc.PRESSURE
    rho_b = 1.004
    p = orc.Problem(dims=dims, tau=0.7, flags=fl, periodic=(0, 0, 1), face_bc=(3, 3, 1, 3, 1, 1),
                    collision=orc.TRT, rho_b=rho_b)
    _, w, _ = orc.lattice()
    f = (w[:, None, None, None] * (rho_b - 1.0)) * (fl == 0)
    g = orc.run(p, f.copy(), 50)
    assert np.abs(g - f).max() < 1e-16
    # the wrong sign or factor would not hold it
    rho, u = orc.macroscopic(p, g)
    assert np.abs(rho[fl == 0] - rho_b).max() < 1e-15 and np.abs(u).max() < 1e-16


# ------------------------------------------------------------ curved walls
def _channel_qw(orc, H, db, dt):
    """Wall distances of a y channel: the bottom wall db below row 0, the top
    wall dt above row H-1, on every link that crosses them."""
    e, _, _ = orc.lattice()
    qw = np.full((19, 1, H, 1), 0.5)
    for i in range(19):
        if e[i, 1] == 1:
            qw[i, 0, 0, 0] = db
        if e[i, 1] == -1:
            qw[i, 0, H - 1, 0] = dt
    return qw


def _poiseuille_error(orc, H, db, dt, coll, curved=True, tau=0.8, F=1e-6):
    p = orc.Problem(dims=(1, H, 1), tau=tau, periodic=(1, 0, 1), collision=coll, force=(F, 0, 0),
                    qw=_channel_qw(orc, H, db, dt) if curved else None)
    f = orc.run(p, orc.zeros(p), 12 * H * H)
    prev = None
    for _ in range(50):
        f = orc.run(p, f, 2000)
        _, u = orc.macroscopic(p, f)
        if prev is not None and np.abs(u - prev).max() < 1e-15:
            break
        prev = u
    nu = (tau - 0.5) / 3
    y = np.arange(H)
    ua = F / (2 * nu) * (y + db) * (H - 1 + dt - y)  # walls at -db and H-1+dt
    return np.abs(u[0, 0, :, 0] - ua).max() / ua.max()


@pytest.mark.parametrize("coll", [0, 1])
@pytest.mark.parametrize("db,dt", [(0.25, 0.25), (0.75, 0.75), (0.1, 0.9), (0.3, 0.6)])
def test_curved_walls_poiseuille_off_grid_second_order(orc, coll, db, dt):
    """Linear interpolated bounce-back (Bouzidi et al.) on a channel whose
    walls sit db below the first and dt above the last fluid row: the steady
    profile converges to the parabola between the true wall positions at
    second order (error ratio ~4 from H = 8 to 16), and is several times
    closer to it than half-way bounce-back, which puts the walls at 1/2."""
    orc.set_threads(os.cpu_count() or 1)
    e8 = _poiseuille_error(orc, 8, db, dt, coll)
    e16 = _poiseuille_error(orc, 16, db, dt, coll)
    half = _poiseuille_error(orc, 16, db, dt, coll, curved=False)
    orc.set_threads(1)
    assert e16 < 8e-3
    assert 3.4 < e8 / e16 < 4.6
    assert half > 3 * e16


def test_curved_walls_at_one_half_are_half_way_bounce_back(orc):
    """Every wall distance 1/2 reduces both interpolations to f*_ibar(x)."""
    rng = np.random.default_rng(21)
    dims = (6, 5, 4)
    fl = _random_flags(rng, dims, 0.3)
    fl[fl == 2] = 1
    kw = dict(dims=dims, tau=0.7, flags=fl, periodic=(1, 0, 0), face_bc=(1,) * 6, collision=1,
              force=(1e-4, 0, 0))
    f = rng.uniform(-1e-2, 1e-2, (19,) + dims[::-1]) * (fl == 0)
    a = orc.step(orc.Problem(**kw), f)
    b = orc.step(orc.Problem(qw=np.full((19,) + dims[::-1], 0.5), **kw), f)
    assert np.array_equal(a, b)


@pytest.mark.parametrize("seed", range(6))
def test_pull_step_matches_push_step_with_curved_walls(orc, seed):
    """Random wall distances on every link into a resting wall or solid cell,
    thin gaps included (where q < 1/2 falls back to half-way bounce-back): the
    pull rule equals the push-and-reflect rule written separately."""
    rng = np.random.default_rng(400 + seed)
    dims = tuple(int(v) for v in rng.integers(3, 6, 3))
    fl = _random_flags(rng, dims, 0.3)
    qw = rng.uniform(0.05, 1.0, (19,) + dims[::-1])
    p = orc.Problem(dims=dims, tau=float(rng.uniform(0.55, 1.5)), flags=fl,
                    periodic=tuple(int(v) for v in rng.integers(0, 2, 3)),
                    face_bc=tuple(int(v) for v in rng.integers(1, 3, 6)), collision=int(seed % 2),
                    magic=float(rng.uniform(0.05, 0.3)), force=tuple(rng.uniform(-1e-3, 1e-3, 3)),
                    wall_u=tuple(rng.uniform(-0.05, 0.05, 3)), qw=qw)
    f = rng.uniform(-1e-2, 1e-2, (19,) + dims[::-1]) * (p.flags == 0)
    for _ in range(3):
        a = orc.step(p, f)
        b = orc.push_step(p, f)
        assert np.abs(a - b).max() < 1e-14
        f = a


def test_step_cells_and_macroscopic_agree_with_step(orc):
    rng = np.random.default_rng(21)
    dims = (6, 5, 7)
    p = orc.Problem(dims=dims, tau=0.7, flags=_random_flags(rng, dims, 0.2),
                    periodic=(1, 0, 1), face_bc=(1, 1, 1, 2, 1, 1), collision=1,
                    force=(1e-4, 0, 0), wall_u=(0.03, 0, 0))
    f = rng.uniform(-1e-2, 1e-2, (19,) + dims[::-1]) * (p.flags == 0)
    g, u_used = orc.step(p, f, return_u=True)
    cells = rng.choice(p.ncells, 40, replace=False)
    got = orc.step_cells(p, f, cells)
    assert np.array_equal(got, g.reshape(19, -1)[:, cells].T)
    rho, u = orc.macroscopic(p, g)
    fluid = p.flags == 0
    assert np.abs((u - u_used)[:, fluid]).max() < 1e-16
    assert np.all(rho[~fluid] == 1.0) and np.all(u[:, ~fluid] == 0.0)


def test_residual_definition(orc):
    rng = np.random.default_rng(4)
    dims = (4, 4, 4)
    p = orc.Problem(dims=dims, tau=0.8, periodic=(1, 1, 1))
    a = rng.uniform(-1e-2, 1e-2, (19,) + dims[::-1])
    assert orc.residual(p, a, a) == 0.0
    assert orc.residual(p, np.zeros_like(a), np.zeros_like(a)) == 0.0
    # u_prev = 0 -> residual exactly 1
    assert abs(orc.residual(p, np.zeros_like(a), a) - 1.0) < 1e-15
    # u_prev = u_cur / 2 -> 1/2
    assert abs(orc.residual(p, a / 2, a) - 0.5) < 1e-15


def test_interval_residual_closed_values(orc):
    """r_k = ||u_n - u_{n-k}|| / (k ||u_n||): zero for equal states, exactly
    1/k from a state at rest, 1/(2k) from half the velocity."""
    rng = np.random.default_rng(41)
    dims = (5, 4, 3)
    p = orc.Problem(dims=dims, tau=0.7, periodic=(1, 1, 1))
    a = rng.uniform(-1e-2, 1e-2, (19,) + dims[::-1])
    z = np.zeros_like(a)
    for k in (1, 2, 50):
        assert orc.interval_residual(p, a, a, k) == 0.0
        assert orc.interval_residual(p, z, z, k) == 0.0
        assert abs(orc.interval_residual(p, z, a, k) - 1.0 / k) < 1e-15
        assert abs(orc.interval_residual(p, a / 2, a, k) - 0.5 / k) < 1e-15


def test_interval_residual_of_uniform_forced_flow(orc):
    """A fully periodic box driven from rest by a uniform force moves as a
    plug.  Its stored momentum grows by exactly F per cell and step, and the
    velocity that step n's collision used (the reported one) carries half of
    that step's force: u_n = (n - 1/2) F.  So the change per step over k
    steps is r = |k F| / (k |u_n|) = 1/(n - 1/2) whatever F and k, and the
    first multiple of k with r < tol follows in closed form.  A dropped
    half-force shift gives 1/n and stops one check earlier below; a dropped
    division by k gives k/(n - 1/2)."""
    dims = (4, 3, 5)
    F = (2e-5, -1e-5, 3e-5)
    for coll in (orc.BGK, orc.TRT):
        p = orc.Problem(dims=dims, tau=0.9, periodic=(1, 1, 1), force=F, collision=coll)
        f = orc.zeros(p)
        g = orc.run(p, f, 30)
        h = orc.run(p, g, 10)
        assert abs(orc.interval_residual(p, g, h, 10) - 1.0 / 39.5) < 1e-10
        assert abs(orc.interval_residual(p, f, h, 40) - 1.0 / 39.5) < 1e-10
        # 1/(n - 1/2) < 1/79.75 first at n = 81 -> the check at 90 (80 if the
        # half-force shift were dropped)
        steps, r, _ = orc.run_to_interval_residual(p, f, 1.0 / 79.75, 10, 1000)
        assert steps == 90 and abs(r - 1.0 / 89.5) < 1e-10, (steps, r)
        steps, r, _ = orc.run_to_interval_residual(p, f, 1.0 / 79.75, 10, 80)
        assert steps == -1 and abs(r - 1.0 / 79.5) < 1e-10


def test_threaded_step_is_identical(orc):
    """The OpenMP split over z planes changes no result bit."""
    from paper_1007_1388_gb300 import workloads as W

    rng = np.random.default_rng(44)
    dims = (9, 7, 11)
    flags = W.random_flags(rng, dims, 0.2)
    p = orc.Problem(dims=dims, tau=0.7, flags=flags, collision=orc.TRT,
                    wall_u=(0.05, 0, 0.01), force=(1e-4, -2e-5, 0))
    f = W.random_pdfs(rng, dims, 1e-2, flags)
    a = orc.run(p, f, 5)
    orc.set_threads(4)
    try:
        b = orc.run(p, f, 5)
    finally:
        orc.set_threads(1)
    assert np.array_equal(a, b)


def test_staggered_mode_stalls_the_one_step_residual(orc):
    """Bounce-back on spheres in a periodic channel excites a period-2
    (staggered) mode that neither BGK nor TRT damps: the one-step velocity
    residual stalls near 1e-4 while the change over two steps is at
    roundoff, i.e. the flow itself is steady.  This fixes the reading of the
    convergence criterion for sphere packings (change per step over an even
    interval)."""
    from paper_1007_1388_gb300 import workloads as W

    n = 16
    fl, F = W.channel_sample(6, n)
    orc.set_threads(os.cpu_count() or 1)
    try:
        for coll in (orc.BGK, orc.TRT):
            p = orc.Problem(dims=(n, n, n), tau=0.8, flags=fl, periodic=(1, 0, 1), force=(F, 0, 0),
                            collision=coll)
            f = orc.run(p, orc.zeros(p), 6000)
            g = orc.step(p, f)
            h = orc.step(p, g)
            one = orc.residual(p, f, g)
            two = orc.residual(p, f, h)
            assert one > 1e-5 and two < 1e-12, (coll, one, two)
            # the change per step over an even interval cancels the mode;
            # over an odd one it does not
            assert orc.interval_residual(p, f, h, 2) < 1e-12
            k3 = orc.step(p, h)
            assert orc.interval_residual(p, f, k3, 3) > 1e-6
    finally:
        orc.set_threads(1)
