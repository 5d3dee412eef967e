"""Pins of the oracle's progressive-mesh criterion (Eq. 13, Sec. 4.2, Fig. 4)
with S > 0 and of the set of blocks it creates, on hand-built states whose
streamed velocities are known in closed form.

Construction: a periodic 24^3 box of 8^3 blocks with only the centre block
meshed, every population at the resting equilibrium of rho = 36 (so that
w_i rho = 12, 2, 1 are exact binary numbers, as are all sums below), and one
post-collision population raised by delta = 1/2.  Pull streaming (Eq. 10,
left) carries it to exactly one cell x, whose moments (Eqs. 4-5) become
rho = 36.5 and j = delta e_i: u = delta e_i / 36.5, every other cell at rest.
The previous velocity is the initial one, 0.  So ||u(0) - u(-1)||_2 is
known, and the criterion must create a block iff that norm exceeds S
(strictly), only when x borders the unmeshed region, and only the unmeshed,
not fully solid blocks that hold a D3Q19 neighbour of x: faces and edges,
never a corner (D3Q19 has no (1, 1, 1) velocity).  A slip in any of those
(comparing ||du||^2 with S, >= for >, a corner block, interior cells
firing, fully solid targets) fails one of these tests."""
import numpy as np
import pytest

from oracle import oracle as O

N, B = 24, 8          # 3 x 3 x 3 blocks
RHO = 36.0
DELTA = 0.5
CENTRE = 1 + 3 * (1 + 3 * 1)


def block_id(bx, by, bz):
    return bx + 3 * (by + 3 * bz)


def lattice_index(e):
    ev, _, _ = O.lattice()
    return [tuple(v) for v in ev].index(tuple(e))


def make(S, ncomp=2, solid_blocks=()):
    ct = np.zeros((N, N, N), dtype=np.uint8)
    for bx, by, bz in solid_blocks:
        ct[bz * B:(bz + 1) * B, by * B:(by + 1) * B, bx * B:(bx + 1) * B] = 1
    rho = np.full((ncomp, N, N, N), RHO)
    amb = np.full(ncomp, RHO)
    s = O.OracleSim(ct, rho, None, amb, ncomp=ncomp, periodic=(1, 1, 1), progressive=1, S=S,
                    g_self=0.0, g_cross=0.0, block=(B, B, B))
    act = np.zeros(27, dtype=np.uint8)
    act[CENTRE] = 1
    s.set_active(act)
    return s


def perturb(s, comp, cell, e, delta=DELTA):
    """Raise the post-collision population of `cell` moving along e (x, y, z
    cell coordinates), which streams to cell + e."""
    f = s.get_f(comp)
    x, y, z = cell
    f[z, y, x, lattice_index(e)] += delta
    s.set_f(comp, f)


def created(s):
    s.step(1)
    return sorted(set(int(b) for b in s.active_blocks()) - {CENTRE})


def test_state_is_exact():
    """The construction itself, by an independent pull of the stored
    populations: x = (15, 12, 12) gets rho = 36.5 and j = (0.5, 0, 0), every
    other cell rho = 36 and j = 0, exactly."""
    s = make(S=1.0)
    perturb(s, 0, (14, 12, 12), (1, 0, 0))
    f = s.get_f(0)  # [z, y, x, i]
    ev, _, _ = O.lattice()
    fin = np.stack([np.roll(f[..., i], shift=(e[2], e[1], e[0]), axis=(0, 1, 2))
                    for i, e in enumerate(ev)], axis=-1)
    rho, j = fin.sum(-1), fin @ ev
    assert rho[12, 12, 15] == RHO + DELTA
    np.testing.assert_array_equal(j[12, 12, 15], [DELTA, 0.0, 0.0])
    rho[12, 12, 15], j[12, 12, 15] = RHO, 0.0
    assert np.all(rho == RHO) and np.all(j == 0.0)


@pytest.mark.parametrize("comp", [0, 1])
def test_threshold_is_strict_on_the_norm(comp):
    """x = (15, 12, 12) borders the +x block; ||du|| = 0.5 / 36.5.  Either
    component's change counts."""
    u = DELTA / (RHO + DELTA)
    target = [block_id(2, 1, 1)]
    for S, expect in ((np.nextafter(u, 0.0), target), (u, []), (np.nextafter(u, 1.0), []),
                      (0.0, target), (u * 0.999, target), (u * 1.001, []), (u * u, target)):
        s = make(S=float(S))
        perturb(s, comp, (14, 12, 12), (1, 0, 0))
        assert created(s) == expect, f"S = {S!r} (||du|| = {u!r})"


def test_targets_are_faces_and_edges_never_corners():
    """x = (15, 15, 15), the centre block's +x+y+z corner cell: its D3Q19
    neighbours reach the three face blocks and the three edge blocks on that
    side, not the corner block (2, 2, 2)."""
    s = make(S=0.0)
    perturb(s, 0, (14, 15, 15), (1, 0, 0))
    expect = sorted([block_id(2, 1, 1), block_id(1, 2, 1), block_id(1, 1, 2),
                     block_id(2, 2, 1), block_id(2, 1, 2), block_id(1, 2, 2)])
    assert created(s) == expect
    assert block_id(2, 2, 2) not in expect


def test_fully_solid_blocks_are_never_created():
    s = make(S=0.0, solid_blocks=[(2, 2, 1)])
    perturb(s, 0, (14, 15, 15), (1, 0, 0))
    expect = sorted([block_id(2, 1, 1), block_id(1, 2, 1), block_id(1, 1, 2),
                     block_id(2, 1, 2), block_id(1, 2, 2)])
    assert created(s) == expect


@pytest.mark.parametrize("x", [(12, 12, 12), (14, 12, 12), (13, 9, 10)])
def test_interior_cells_create_nothing(x):
    """A cell whose D3Q19 neighbours all lie in the meshed block fires (its
    velocity changes by far more than S) but borders no unmeshed block."""
    s = make(S=0.0)
    perturb(s, 0, (x[0] - 1, x[1], x[2]), (1, 0, 0))
    assert created(s) == []


def test_density_only_change_is_not_seen():
    """The symmetric counter-case: the two populations arriving at the
    border cell x = (15, 12, 12) along +y and -y both rise by delta.  Its
    density changes by 2 delta, its velocity not at all, so Eq. 13 (a
    velocity criterion) misses the change even at S = 0, and nothing is
    created.  Raising only one of them moves x and creates the +x block."""
    s = make(S=0.0)
    perturb(s, 0, (15, 11, 12), (0, 1, 0))
    perturb(s, 0, (15, 13, 12), (0, -1, 0))
    assert created(s) == []
    s = make(S=0.0)
    perturb(s, 0, (15, 11, 12), (0, 1, 0))
    assert created(s) == [block_id(2, 1, 1)]
