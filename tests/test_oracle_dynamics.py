"""Pins of the oracle's full time step: conservation laws, the resting
ambient as a fixed point, the Poiseuille closed form, Laplace's law,
liquid-vapour coexistence, and the progressive mesh reproducing the static
mesh exactly (Sec. 4.1-4.3, Eq. 13)."""
import numpy as np
import pytest

from oracle import oracle as O
from paper_1510_03560_gb300 import workloads as W


def sim_of(case, **over):
    p = dict(case["params"])
    p.update(over)
    return O.OracleSim(case["cell_type"], case["rho_init"], case["u_init"], case["rho_amb"], **p)


def porous_periodic(n=24, seed=5, frac=0.2, ncomp=2):
    solid = W.spheres_mask((n, n, n), seed, frac, (2.0, 4.0), 0)
    rng = np.random.default_rng(seed)
    ct = solid.astype(np.uint8)
    rho = np.empty((ncomp, n, n, n))
    rho[0] = W.RHO_VAP * (1 + 0.05 * rng.standard_normal((n, n, n)))
    blob = rng.uniform(size=(n, n, n)) < 0.15
    rho[0][blob] = W.RHO_LIQ
    if ncomp == 2:
        rho[1] = np.where(blob, 0.01, 1.0)
    amb = np.array([W.RHO_VAP, 1.0][:ncomp])
    params = dict(W.PHYSICS, ncomp=ncomp, periodic=(1, 1, 1), progressive=0,
                  g_ads=(-0.2, 0.0), grav=(0.0, 0.0, -1e-5), block=(8, 8, 8))
    return ct, rho, amb, params


def test_mass_conserved_closed_box():
    """Streaming with halfway bounce-back and the forced collision conserve
    each component's mass (closed box with solids, static mesh)."""
    ct, rho, amb, params = porous_periodic()
    s = O.OracleSim(ct, rho, None, amb, **params)
    m0 = s.mass()
    s.step(30)
    np.testing.assert_allclose(s.mass(), m0, rtol=1e-13)
    case = W.drop_in_box(progressive=0)
    s = sim_of(case)
    m0 = s.mass()
    s.step(30)
    np.testing.assert_allclose(s.mass(), m0, rtol=1e-13)


def momentum(s):
    e, _, _ = O.lattice()
    return sum(np.einsum("zyxi,ia->a", s.get_f(a), e) for a in range(s.ncomp))


def test_momentum_conserved_periodic():
    """Without solids and gravity the interaction forces of Eqs. 8-9 sum to
    zero over a periodic box, so total momentum is conserved."""
    ct, rho, amb, params = porous_periodic(n=16, frac=0.0)
    params.update(grav=(0.0, 0.0, 0.0), g_ads=(0.0, 0.0))
    u = np.zeros((2, 3) + ct.shape)
    u[:, 0] = 0.01
    s = O.OracleSim(ct, rho, u, amb, **params)
    p0 = momentum(s)
    s.step(20)
    scale = float(np.abs(rho).sum())
    np.testing.assert_allclose(momentum(s), p0, rtol=0, atol=1e-13 * scale)


def test_resting_ambient_is_fixed_point():
    """A uniform ambient at rest next to arbitrary solids stays at rest
    (neutral-wall psi, bounce-back, buoyancy gravity and the
    ambient-excess adhesion all vanish there)."""
    ct, rho, amb, params = porous_periodic(n=16)
    amb = np.array([fixed_point(W.RHO_VAP), fixed_point(1.0)])
    rho[0] = amb[0]
    rho[1] = amb[1]
    params.update(periodic=(1, 0, 1), g_ads=(-0.2, 0.0), rho_ref=tuple(amb))
    s = O.OracleSim(ct, rho, None, amb, **params)
    f0 = [s.get_f(a) for a in range(2)]
    s.step(20)
    fluid = ct == 0
    for a in range(2):
        r, ux, uy, uz = s.macro(a)
        assert np.all(ux[fluid] == 0) and np.all(uy[fluid] == 0) and np.all(uz[fluid] == 0)
        assert np.all(r[fluid] == amb[a])
        np.testing.assert_array_equal(s.get_f(a)[fluid], f0[a][fluid])


@pytest.mark.parametrize("H,steps", [(8, 2000), (16, 3000), (32, 8000)])
def test_poiseuille(H, steps):
    """Body-force-driven flow between halfway bounce-back plates: the steady
    profile is exactly parabolic (second difference -g/nu) and its
    deviation from g (z - z0)(z0 + H - z) / (2 nu), walls half-way between
    cells, shrinks at second order in 1/H."""
    gx, nu = 1e-6, 1.0 / 6.0
    case = W.channel(H=H, nxy=4, gx=gx, block=(4, 4, 8))
    nz = case["cell_type"].shape[0]
    z = np.arange(nz)
    ua = gx / (2 * nu) * (z - 0.5) * (H + 0.5 - z)
    ua[0] = 0
    ua[H + 1:] = 0
    u = np.zeros((1, 3) + case["cell_type"].shape)
    u[0, 0] = ua[:, None, None]
    s = O.OracleSim(case["cell_type"], case["rho_init"], u, case["rho_amb"], **case["params"])
    s.step(steps)
    prof = s.macro(0)[1][1:H + 1, 2, 2]
    d2 = prof[2:] - 2 * prof[1:-1] + prof[:-2]
    np.testing.assert_allclose(d2 * nu / gx, -1.0, atol=1e-5)
    exact = ua[1:H + 1]
    err = np.abs(prof - exact).max() / exact.max()
    assert err * H * H < 0.4


def test_laplace_law():
    """Single-component droplets: the pressure jump between the bulk phases
    (EOS at the measured bulk densities) is linear in 1/R with a near-zero
    intercept (Laplace's law)."""
    inv_r, dp = [], []
    n = 32
    for R in (8.0, 9.0, 10.0, 11.0, 12.0):
        case = W.droplet(n=n, R=R, rho_vap=0.42)
        s = sim_of(case)
        s.step(1000)
        r = s.macro(0)[0]
        m = n // 2
        rin, rout = r[m, m, m], r[0, 0, 0]
        V = (r.sum() - rout * r.size) / (rin - rout)
        inv_r.append(1.0 / (3 * V / (4 * np.pi)) ** (1 / 3))
        dp.append(O.pressure(rin) - O.pressure(rout))
    inv_r, dp = np.array(inv_r), np.array(dp)
    slope, icpt = np.polyfit(inv_r, dp, 1)
    fit = slope * inv_r + icpt
    r2 = 1 - ((dp - fit) ** 2).sum() / ((dp - dp.mean()) ** 2).sum()
    assert r2 > 0.99
    assert slope > 0
    assert abs(icpt) < 0.05 * dp.max()


def test_flat_interface_coexistence():
    """A flat liquid slab relaxes to bulk densities near the Maxwell values
    (within 5 % liquid, 10 % vapour), and beta = 1.16 brings the vapour
    closer to them than beta = 1 (the purpose of the beta mixing of Eq. 8)."""
    errs = {}
    for beta in (1.0, 1.16):
        case = W.slab(nxy=8, nz=64)
        s = sim_of(case, beta=beta)
        s.step(3000)
        r = s.macro(0)[0]
        rl, rg = r[32, 4, 4], r[0, 4, 4]
        errs[beta] = (abs(rl - W.RHO_LIQ) / W.RHO_LIQ, abs(rg - W.RHO_VAP) / W.RHO_VAP)
    assert errs[1.16][0] < 0.05 and errs[1.16][1] < 0.10
    assert errs[1.16][1] < errs[1.0][1]


def test_hydrostatic_column_physical_velocity():
    """Closed column under a body force rho g: it comes to rest, and the
    reported velocity u + F/(2 rho) vanishes (the bare Eq. 5 velocity
    settles at -F/(2 rho), a thousand times larger than the bound)."""
    case = W.channel(H=14, nxy=4, gx=0.0, block=(4, 4, 8))
    p = dict(case["params"], grav=(0.0, 0.0, -1e-4))
    s = O.OracleSim(case["cell_type"], case["rho_init"], None, case["rho_amb"], **p)
    s.step(3000)
    r, ux, uy, uz = s.macro(0)
    fluid = case["cell_type"] == 0
    half_kick = 1e-4 / 2  # |F| / (2 rho) with F = rho g
    assert np.abs(uz[fluid]).max() < 1e-3 * half_kick
    assert r[1, 2, 2] > r[14, 2, 2]  # denser at the bottom


def test_held_cells_keep_their_state():
    case = W.porous_injection(n=(32, 32, 32), seed=3, inlet=8, x_free=4, r_range=(2.0, 4.0))
    s = sim_of(case, progressive=0)
    held = case["cell_type"] == W.HELD
    f0 = [s.get_f(a)[held] for a in range(2)]
    s.step(10)
    for a in range(2):
        np.testing.assert_array_equal(s.get_f(a)[held], f0[a])


def fixed_point(r):
    """Density reproduced exactly by summing its own resting equilibrium."""
    _, w, _ = O.lattice()
    for _ in range(50):
        s = 0.0
        for wi in w:
            s += wi * r
        if s == r:
            return r
        r = s
    raise AssertionError("no fixed point")


def state_with_ambient(s, amb, block):
    """Post-collision populations, unmeshed cells shown at the ambient
    equilibrium and solid cells zeroed."""
    nz, ny, nx = s.shape
    bx, by, bz = block
    act = np.zeros(s.nblock, bool)
    act[s.active_blocks()] = True
    cells = act.reshape(nz // bz, ny // by, nx // bx)
    cells = np.repeat(np.repeat(np.repeat(cells, bz, 0), by, 1), bx, 2)
    _, w, _ = O.lattice()
    out = []
    for a in range(s.ncomp):
        f = np.where(cells[..., None], s.get_f(a), w * amb[a])
        out.append(f)
    return np.stack(out)


def test_progressive_equals_static():
    """With S = 0 and a bit-stationary ambient (new blocks start at rest in it), meshing blocks only
    where Eq. 13 fires reproduces the static mesh exactly at every step,
    while far blocks stay unmeshed for a while."""
    amb = (fixed_point(W.f32(W.RHO_VAP)), fixed_point(1.0))
    block = (4, 4, 4)
    sims = []
    for prog in (1, 0):
        case = W.blob(n=24, block=block, S=0.0, progressive=prog)
        rho = case["rho_init"].astype(np.float64)
        for a in range(2):
            rho[a][rho[a] == np.float32(case["rho_amb"][a])] = amb[a]
        p = dict(case["params"], rho_ref=amb)
        sims.append(O.OracleSim(case["cell_type"], rho, None, np.array(amb), **p))
    prog, stat = sims
    ct = case["cell_type"]
    counts = []
    for _ in range(24):
        prog.step(1)
        stat.step(1)
        a = state_with_ambient(prog, amb, block)
        b = state_with_ambient(stat, amb, block)
        a[:, ct == 1] = 0
        b[:, ct == 1] = 0
        np.testing.assert_array_equal(a, b)
        counts.append(len(prog.active_blocks()))
    assert counts[0] < prog.nblock // 4
    assert counts == sorted(counts)
    assert counts[-1] > counts[0]


def test_streaming_brute_force():
    """One force-free tau = 1 step on random populations equals a direct
    array-shift evaluation of pull streaming with halfway bounce-back
    followed by relaxation to equilibrium (Eqs. 1, 2, 4, 5)."""
    n = 8
    rng = np.random.default_rng(11)
    ct = (rng.uniform(size=(n, n, n)) < 0.2).astype(np.uint8)
    rho = np.ones((1, n, n, n))
    params = dict(W.PHYSICS, ncomp=1, periodic=(1, 1, 1), progressive=0, g_self=0.0,
                  g_cross=0.0, grav=(0.0, 0.0, 0.0), block=(4, 4, 4))
    s = O.OracleSim(ct, rho, None, np.array([1.0]), **params)
    e, w, opp = O.lattice()
    f = rng.uniform(0.01, 0.1, size=(n, n, n, 19))
    s.set_f(0, f)
    s.step(1)
    got = s.get_f(0)
    solid = ct == 1
    fin = np.empty_like(f)
    for i in range(19):
        shift = (int(e[i, 2]), int(e[i, 1]), int(e[i, 0]))
        moved = np.roll(f[..., i], shift, axis=(0, 1, 2))
        from_solid = np.roll(solid, shift, axis=(0, 1, 2))
        fin[..., i] = np.where(from_solid, f[..., opp[i]], moved)
    r = fin.sum(-1)
    u = np.einsum("zyxi,ia->zyxa", fin, e) / r[..., None]
    for idx in zip(*np.nonzero(~solid)):
        np.testing.assert_allclose(got[idx], O.feq(r[idx], u[idx]), rtol=1e-13, atol=1e-16)
